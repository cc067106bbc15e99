// Adaptive octree shared by the adaptive kernels (3D).
//
// Boxes are numbered level by level; inside a level they are in Morton order
// of their integer coordinates (bit b of x, y, z at key bits 3b, 3b+1, 3b+2),
// so a box is found by binary search of its code among the level's boxes.
// Points are sorted by their Morton code at the deepest level, which makes
// the sources (targets) of every box a contiguous range [s0, s1) ([t0, t1)).
//
// "Adjacent" means the closed boxes touch or coincide.  The interaction lists
// of a box B of level l (parent P(B)) are
//   U(B), B a leaf: leaves adjacent to B, B included                 (P2P)
//   V(B), l >= 2:   children of the boxes adjacent to P(B) that are not
//                   adjacent to B                                    (M2L)
//   W(B), B a leaf: boxes C finer than B with P(C) adjacent to B and C
//                   not adjacent to B                                (M2P)
//   X(B), l >= 2:   leaves A coarser than B adjacent to P(B) and not
//                   adjacent to B                                    (P2L)
// The kernels enumerate them on the fly from these lookups; nothing is stored.
#pragma once

#include "fmm_internal.cuh"

#define FMM_MAX_ADEPTH 10  // 30-bit Morton codes

struct ATree {
  const uint32_t* key;  // Morton code of each box at its own level
  const int* lev;
  const int* par;
  const int* child;     // 8 per box (octant x | y<<1 | z<<2), -1 if absent
  const int* s0;
  const int* s1;
  const int* t0;
  const int* t1;
  const int* leaf;
  const int* grid;  // dense index of levels 0..grid_levels: grid[(8^l - 1)/7 + code] = box or -1
  int grid_levels;
  int loff[FMM_MAX_ADEPTH + 2];  // first box of each level; loff[maxlev+1] = boxes
  int maxlev;
};

#define FMM_AGRID_LEVELS 7  // dense index down to level 7: sum 8^l = 2,396,745 entries

__host__ __device__ inline int64_t agrid_offset(int l) { return (((int64_t)1 << (3 * l)) - 1) / 7; }

__host__ __device__ inline uint32_t morton3(int x, int y, int z, int l) {
  uint32_t k = 0;
  for (int b = l - 1; b >= 0; --b)
    k = (k << 3) | (uint32_t)((x >> b) & 1) | ((uint32_t)((y >> b) & 1) << 1) |
        ((uint32_t)((z >> b) & 1) << 2);
  return k;
}

__host__ __device__ inline void demorton3(uint32_t k, int l, int* c) {
  c[0] = c[1] = c[2] = 0;
  for (int b = 0; b < l; ++b) {
    c[0] |= (int)((k >> (3 * b)) & 1) << b;
    c[1] |= (int)((k >> (3 * b + 1)) & 1) << b;
    c[2] |= (int)((k >> (3 * b + 2)) & 1) << b;
  }
}

// index of the box of level l at coordinates c, or -1
__device__ inline int alookup(const ATree& t, int l, const int* c) {
  const int n = 1 << l;
  if (c[0] < 0 || c[1] < 0 || c[2] < 0 || c[0] >= n || c[1] >= n || c[2] >= n) return -1;
  if (l > t.maxlev) return -1;
  const uint32_t k = morton3(c[0], c[1], c[2], l);
  if (l <= t.grid_levels) return t.grid[agrid_offset(l) + k];
  int lo = t.loff[l], hi = t.loff[l + 1];
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (t.key[mid] < k) lo = mid + 1;
    else hi = mid;
  }
  return (lo < t.loff[l + 1] && t.key[lo] == k) ? lo : -1;
}

// closed boxes (la, ca) and (lb, cb) touch or overlap
__device__ inline bool aadjacent(int la, const int* ca, int lb, const int* cb) {
  const int m = la > lb ? la : lb;
  for (int k = 0; k < 3; ++k) {
    const int a0 = ca[k] << (m - la), a1 = (ca[k] + 1) << (m - la);
    const int b0 = cb[k] << (m - lb), b1 = (cb[k] + 1) << (m - lb);
    if (a0 > b1 || b0 > a1) return false;
  }
  return true;
}

__device__ inline void abox(const ATree& t, int b, int* l, int* c) {
  *l = t.lev[b];
  demorton3(t.key[b], *l, c);
}

// centre and side of a box, in the same operations as the uniform tree:
// s = size / 2^l, c_k = lo_k + (coord_k + 1/2) s
__device__ inline void abox_center(const Geom* g, int l, const int* bc, double* c, double* s) {
  const double sl = __dmul_rn(g->size, __longlong_as_double((long long)(1023 - l) << 52));
  for (int k = 0; k < 3; ++k) c[k] = __dadd_rn(g->lo[k], __dmul_rn((double)bc[k] + 0.5, sl));
  *s = sl;
}

// host-side bound on the number of boxes of an adaptive tree over n points
inline int64_t adaptive_box_bound(int64_t n, int max_leaf, int depth) {
  int64_t splits_cap = n / ((int64_t)max_leaf + 1);
  int64_t nb = 1, lvl = 1;
  for (int l = 0; l < depth; ++l) {
    const int64_t splits = lvl < splits_cap ? lvl : splits_cap;
    lvl = 8 * splits < n ? 8 * splits : n;  // boxes of level l+1 (none empty)
    nb += lvl;
    if (lvl == 0) break;
  }
  return nb;
}
