// Uniform-tree construction on the device: root geometry, leaf binning, a
// stable LSD radix sort of (leaf key, original index), leaf ranges, and the
// gather of positions/weights into leaf order (SoA).
//
// Leaf boxes are numbered lexicographically, x fastest.  A point's leaf
// coordinate is floor((x - lo) / s_L) with s_L = size / 2^L, evaluated with
// round-to-nearest operations only, so the binning is reproducible.
#include <algorithm>

#include "adaptive.cuh"
#include "fmm_internal.cuh"

namespace {

constexpr int kRsBlock = 1024;

__device__ void set_leaf_side(Geom* g, int L) {
  g->s_leaf = __ddiv_rn(g->size, (double)(1 << L));
  g->inv_s_leaf = 1.0 / g->s_leaf;
  g->m2l_count = 0;
  g->p2p_pairs = 0;
}

__global__ void k_geom_fixed(Geom* g, double lo0, double lo1, double lo2, double size, int L) {
  g->lo[0] = lo0;
  g->lo[1] = lo1;
  g->lo[2] = lo2;
  g->size = size;
  g->flag = 0;
  set_leaf_side(g, L);
}

// per-block min/max over the sources and targets (bounding cube of the root)
template <int D>
__global__ void k_bbox_partial(int64_t ns, const double* __restrict__ src, int64_t nt,
                               const double* __restrict__ tgt, double* out) {
  __shared__ double smin[D][256], smax[D][256];
  double mn[D], mx[D];
  for (int k = 0; k < D; ++k) {
    mn[k] = INFINITY;
    mx[k] = -INFINITY;
  }
  const int64_t n = ns + nt;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double* x = i < ns ? src + i * D : tgt + (i - ns) * D;
    for (int k = 0; k < D; ++k) {
      mn[k] = fmin(mn[k], x[k]);
      mx[k] = fmax(mx[k], x[k]);
    }
  }
  for (int k = 0; k < D; ++k) {
    smin[k][threadIdx.x] = mn[k];
    smax[k][threadIdx.x] = mx[k];
  }
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < D; ++k) {
        smin[k][threadIdx.x] = fmin(smin[k][threadIdx.x], smin[k][threadIdx.x + s]);
        smax[k][threadIdx.x] = fmax(smax[k][threadIdx.x], smax[k][threadIdx.x + s]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < D; ++k) {
      out[(blockIdx.x * 2 + 0) * 3 + k] = smin[k][0];
      out[(blockIdx.x * 2 + 1) * 3 + k] = smax[k][0];
    }
}

// root = cube with corner at the minimum and side = the largest extent
template <int D>
__global__ void k_bbox_final(int nblk, const double* part, Geom* g, int L) {
  if (threadIdx.x != 0) return;
  double mn[3] = {0, 0, 0}, mx[3] = {0, 0, 0};
  for (int k = 0; k < D; ++k) {
    mn[k] = INFINITY;
    mx[k] = -INFINITY;
  }
  for (int b = 0; b < nblk; ++b)
    for (int k = 0; k < D; ++k) {
      mn[k] = fmin(mn[k], part[(b * 2 + 0) * 3 + k]);
      mx[k] = fmax(mx[k], part[(b * 2 + 1) * 3 + k]);
    }
  double size = 0.0;
  for (int k = 0; k < D; ++k) size = fmax(size, mx[k] - mn[k]);
  if (!(size > 0.0) || !isfinite(size)) size = 1.0;
  for (int k = 0; k < 3; ++k) g->lo[k] = (k < D && isfinite(mn[k])) ? mn[k] : 0.0;
  g->size = size;
  g->flag = 0;
  set_leaf_side(g, L);
}

}  // namespace

// (x - lo) / s rounded as an IEEE division.  The product with 1/s differs
// from the quotient by at most an ulp, which matters only when the quotient is
// within an ulp of an integer (a box face); those rare points take the exact
// division, so every point lands in the same leaf as with the division.
__device__ __forceinline__ double leaf_coord(double x, double lo, double s, double inv_s) {
  const double d = __dsub_rn(x, lo);
  const double t = d * inv_s;
  if (fabs(t - rint(t)) < 1e-6) return __ddiv_rn(d, s);
  return t;
}

namespace {

// leaf key of every point + per-leaf counts; vals = identity
template <int D>
__global__ void k_bin(int64_t n, const double* __restrict__ x, const Geom* __restrict__ g, int L,
                      uint32_t* __restrict__ keys, int* __restrict__ vals,
                      int* __restrict__ counts, Geom* gflag) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int nl = 1 << L;
  const double s = g->s_leaf, inv_s = g->inv_s_leaf;
  const float inv_sf = (float)inv_s;
  uint32_t key = 0;
  bool bad = false;
  for (int k = D - 1; k >= 0; --k) {
    const double xv = x[i * D + k];
    // float estimate, off by far less than 1e-3 box widths; only points that
    // close to a box face take the FP64 path (identical to the division)
    const float tf = (float)(xv - g->lo[k]) * inv_sf;  // relative error ~2^-23 of t <= 2^L
    int b;
    if (tf >= 0.001f && tf <= (float)nl - 0.001f && fabsf(tf - rintf(tf)) > 0.001f) {
      b = min((int)tf, nl - 1);
    } else {
      const double t = leaf_coord(xv, g->lo[k], s, inv_s);
      if (!(t >= 0.0) || t > (double)nl) bad = true;
      b = (t >= 0.0) ? (int)fmin(floor(t), (double)(nl - 1)) : 0;  // NaN -> 0
    }
    key = key * (uint32_t)nl + (uint32_t)b;
  }
  if (bad) atomicOr(&gflag->flag, 1);
  keys[i] = key;
  vals[i] = (int)i;
  atomicAdd(&counts[key], 1);
}

// ---- exclusive scan of an int array (three small kernels) -----------------
__device__ int block_exclusive_scan(int v, int* smem, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int nw = blockDim.x >> 5;
    int s = lane < nw ? smem[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    smem[lane] = s;
  }
  __syncthreads();
  int incl = x + (wid > 0 ? smem[wid - 1] : 0);
  if (total) *total = smem[(blockDim.x >> 5) - 1];
  __syncthreads();
  return incl - v;
}

__global__ void k_scan_chunks(const int* __restrict__ in, int* __restrict__ out, int64_t n,
                              int* __restrict__ sums) {
  __shared__ int sm[32];
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int v = i < n ? in[i] : 0;
  int tot;
  int ex = block_exclusive_scan(v, sm, &tot);
  if (i < n) out[i] = ex;
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_top(int* sums, int n) {
  // one block: each thread scans a contiguous segment
  __shared__ int sm[32];
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int b = threadIdx.x * per;
  int loc = 0;
  for (int k = 0; k < per && b + k < n; ++k) loc += sums[b + k];
  int ex = block_exclusive_scan(loc, sm, nullptr);
  int run = ex;
  for (int k = 0; k < per && b + k < n; ++k) {
    int v = sums[b + k];
    sums[b + k] = run;
    run += v;
  }
}

__global__ void k_scan_add(int* __restrict__ out, int64_t n, const int* __restrict__ sums,
                           int* __restrict__ total_out, const int* __restrict__ in_last) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] += sums[blockIdx.x];
  if (total_out && i == n - 1) *total_out = out[i] + *in_last;
}

// ---- stable LSD radix sort, 8 bits per pass --------------------------------
__global__ void k_rs_hist(const uint32_t* __restrict__ keys, int n, int shift,
                          int* __restrict__ hist, int nblk) {
  __shared__ int h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  int i = blockIdx.x * kRsBlock + threadIdx.x;
  if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
  __syncthreads();
  for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b * nblk + blockIdx.x] = h[b];
}

__global__ void k_rs_scatter(const uint32_t* __restrict__ kin, const int* __restrict__ vin,
                             uint32_t* __restrict__ kout, int* __restrict__ vout, int n, int shift,
                             const int* __restrict__ hist_ex, int nblk) {
  __shared__ unsigned short wc[32][256];
  for (int i = threadIdx.x; i < 32 * 256; i += blockDim.x) (&wc[0][0])[i] = 0;
  __syncthreads();
  const int i = blockIdx.x * kRsBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const bool valid = i < n;
  uint32_t key = valid ? kin[i] : 0u;
  int val = valid ? vin[i] : 0;
  const unsigned dig = valid ? ((key >> shift) & 255u) : 256u;
  const unsigned peers = __match_any_sync(0xffffffffu, dig);
  const int rank = __popc(peers & ((1u << lane) - 1u));
  if (valid && rank == 0) wc[wid][dig] = (unsigned short)__popc(peers);
  __syncthreads();
  if (threadIdx.x < 256) {
    unsigned run = 0;
    for (int w = 0; w < 32; ++w) {
      unsigned c = wc[w][threadIdx.x];
      wc[w][threadIdx.x] = (unsigned short)run;
      run += c;
    }
  }
  __syncthreads();
  if (valid) {
    int pos = hist_ex[dig * nblk + blockIdx.x] + wc[wid][dig] + rank;
    kout[pos] = key;
    vout[pos] = val;
  }
}

template <int D>
__global__ void k_gather(int n, const int* __restrict__ order, const double* __restrict__ x,
                         const double* __restrict__ w, double* __restrict__ o0,
                         double* __restrict__ o1, double* __restrict__ o2,
                         double* __restrict__ ow, int* __restrict__ perm) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int j = order[i];
  perm[i] = j;
  o0[i] = x[(int64_t)j * D + 0];
  o1[i] = x[(int64_t)j * D + 1];
  if (D == 3) o2[i] = x[(int64_t)j * D + 2];
  if (w) ow[i] = w[j];
}

// FP32 path (d = 3): sorted points as float4 (x - c_own)/s and weight, c_own
// the centre of the point's own leaf.
// The leaf of sorted point i is its sorted key; (x - c)/s = (x - lo)/s - (b + 1/2).
__global__ void k_gather_rel(int n, const int* __restrict__ order,
                             const uint32_t* __restrict__ keys, const double* __restrict__ x,
                             const double* __restrict__ w, const Geom* __restrict__ g, int L,
                             float4* __restrict__ out, int* __restrict__ perm) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int j = order[i];
  perm[i] = j;
  const uint32_t nl = 1u << L;
  uint32_t key = keys[i];
  const double inv_s = g->inv_s_leaf;
  float u[3];
  for (int k = 0; k < 3; ++k) {
    const uint32_t b = key % nl;
    key /= nl;
    const double t = (x[(int64_t)j * 3 + k] - g->lo[k]) * inv_s;
    u[k] = (float)(t - ((double)b + 0.5));
  }
  out[i] = make_float4(u[0], u[1], u[2], w ? (float)w[j] : 0.f);
}

// ---- adaptive octree (adaptive.cuh) ----------------------------------------
// Morton code of every point at the deepest level D, from the same leaf
// coordinates as the uniform binning (leaf side = root / 2^D).
__global__ void k_amorton(int64_t n, const double* __restrict__ x, const Geom* __restrict__ g,
                          int D, uint32_t* __restrict__ keys, int* __restrict__ vals, Geom* gflag) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int nl = 1 << D;
  const double s = g->s_leaf, inv_s = g->inv_s_leaf;
  int bc[3];
  bool bad = false;
  for (int k = 0; k < 3; ++k) {
    const double t = leaf_coord(x[i * 3 + k], g->lo[k], s, inv_s);
    if (!(t >= 0.0) || t > (double)nl) bad = true;
    bc[k] = (t >= 0.0) ? (int)fmin(floor(t), (double)(nl - 1)) : 0;  // NaN -> 0
  }
  if (bad) atomicOr(&gflag->flag, 1);
  keys[i] = morton3(bc[0], bc[1], bc[2], D);
  vals[i] = (int)i;
}

__global__ void k_atree_root(int* lev, int* par, uint32_t* key, int* s0, int* s1, int* t0,
                             int* t1, int ns, int nt, int* dlo, int nlo) {
  for (int l = 0; l < nlo; ++l) dlo[l] = l == 0 ? 0 : 1;  // level offsets: the root alone
  dlo[nlo] = 0;                                          // overflow flag
  lev[0] = 0;
  par[0] = -1;
  key[0] = 0;
  s0[0] = 0;
  s1[0] = ns;
  t0[0] = 0;
  t1[0] = nt;
}

// sources as (hi, lo) float pairs: hi = fl(x), lo = fl(x - hi), weight in hi.w
__global__ void k_split_points(int64_t n, const double* __restrict__ x0,
                               const double* __restrict__ x1, const double* __restrict__ x2,
                               const double* __restrict__ w, float4* __restrict__ hi,
                               float4* __restrict__ lo) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float h0 = (float)x0[i], h1 = (float)x1[i], h2 = (float)x2[i];
  hi[i] = make_float4(h0, h1, h2, (float)w[i]);
  lo[i] = make_float4((float)(x0[i] - (double)h0), (float)(x1[i] - (double)h1),
                      (float)(x2[i] - (double)h2), 0.f);
}

// per-level coordinate bounds of the boxes of levels >= 2 (the windows of the
// adaptive tensor-core M2L): bnd[6 l + k] = min, bnd[6 l + 3 + k] = max
__global__ void k_abounds_init(int* bnd, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) bnd[i] = (i % 6) < 3 ? 0x7fffffff : -1;
}
__global__ void k_abounds(const int* __restrict__ dlo, int D, const int* __restrict__ lev,
                          const uint32_t* __restrict__ key, int* __restrict__ bnd) {
  // boxes are stored level by level, so a warp mostly holds one level: reduce
  // over the lanes of each level first, one atomic per level and warp
  const int b = blockIdx.x * blockDim.x + threadIdx.x;  // the grid covers whole warps
  int l = -1, c[3] = {0, 0, 0};
  if (b < dlo[D + 1] && lev[b] >= 2) {
    l = lev[b];
    demorton3(key[b], l, c);
  }
  const unsigned grp = __match_any_sync(0xffffffffu, l);
  if (l < 0) return;
  const bool lead = (threadIdx.x & 31) == __ffs(grp) - 1;
  for (int k = 0; k < 3; ++k) {
    const int mn = __reduce_min_sync(grp, c[k]), mx = __reduce_max_sync(grp, c[k]);
    if (lead) {
      atomicMin(&bnd[6 * l + k], mn);
      atomicMax(&bnd[6 * l + 3 + k], mx);
    }
  }
}

// dense index of the coarse levels: grid[(8^l - 1)/7 + code] = box
__global__ void k_agrid_fill(int nbox, int glev, const uint32_t* __restrict__ key,
                             const int* __restrict__ lev, int* __restrict__ grid) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox || lev[b] > glev) return;
  grid[agrid_offset(lev[b]) + key[b]] = b;
}

// first position in sorted[lo, hi) whose code is >= v
__device__ inline int lower_bound_u32(const uint32_t* a, int lo, int hi, uint32_t v) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// A box's child ranges are the boundaries of its octants 1..7 in the sorted
// source and target codes: fourteen binary searches, one per lane of a group
// of 16 lanes (lanes 0..6 sources, 8..14 targets), so that a level's kernels
// wait for one search's chain of dependent loads, not fourteen.  Every lane of
// the group gets all boundaries sb[0..8], tb[0..8] by shuffles.
constexpr int kBoxLanes = 16;
__device__ __forceinline__ void child_bounds_group(const uint32_t* skey, const uint32_t* tkey,
                                                   bool live, uint32_t key, int l, int D, int s0,
                                                   int s1, int t0, int t1, int* sb, int* tb) {
  const int k = threadIdx.x & (kBoxLanes - 1);
  int v = 0;
  if (live && k != 7 && k != 15) {
    const int ci = (k & 7) + 1;
    const uint32_t c = ((key << 3) | (uint32_t)ci) << (3 * (D - l - 1));
    v = k < 8 ? lower_bound_u32(skey, s0, s1, c) : lower_bound_u32(tkey, t0, t1, c);
  }
  sb[0] = s0;
  tb[0] = t0;
#pragma unroll
  for (int ci = 1; ci < 8; ++ci) {
    sb[ci] = __shfl_sync(0xffffffffu, v, ci - 1, kBoxLanes);
    tb[ci] = __shfl_sync(0xffffffffu, v, ci + 7, kBoxLanes);
  }
  sb[8] = s1;
  tb[8] = t1;
}

// split decision and number of non-empty children of every box of level l,
// boxes dlo[l] .. dlo[l+1] (level offsets kept on the device); 16 lanes a box
__global__ void k_atree_split(const int* __restrict__ dlo, int l, int D, int max_leaf,
                              const uint32_t* __restrict__ key, const int* __restrict__ s0,
                              const int* __restrict__ s1, const int* __restrict__ t0,
                              const int* __restrict__ t1, const uint32_t* __restrict__ skey,
                              const uint32_t* __restrict__ tkey, int* __restrict__ leaf,
                              int* __restrict__ child, int* __restrict__ nch) {
  const int b0 = dlo[l], b1 = dlo[l + 1];
  const int b = b0 + (int)((blockIdx.x * blockDim.x + threadIdx.x) / kBoxLanes);
  const int k = threadIdx.x & (kBoxLanes - 1);
  const bool live = b < b1;
  bool split = false;
  int bs0 = 0, bs1 = 0, bt0 = 0, bt1 = 0;
  uint32_t bkey = 0;
  if (live) {
    bs0 = s0[b], bs1 = s1[b], bt0 = t0[b], bt1 = t1[b];
    bkey = key[b];
    split = (bs1 - bs0) + (bt1 - bt0) > max_leaf && l < D;
    if (k < 8) child[8 * b + k] = -1;
    if (k == 0) leaf[b] = split ? 0 : 1;
  }
  int sb[9], tb[9];  // every lane of the block reaches the shuffles
  child_bounds_group(skey, tkey, live && split, bkey, l, D, bs0, bs1, bt0, bt1, sb, tb);
  if (live && k == 0) {
    int n = 0;
    if (split)
      for (int ci = 0; ci < 8; ++ci) n += (sb[ci + 1] > sb[ci] || tb[ci + 1] > tb[ci]) ? 1 : 0;
    nch[b - b0] = n;
  }
}

// create the children of level l's split boxes at dlo[l+1] + scan[b - b0]
// (scan[nscan] = the children of the level, the counts past the level being
// zero) and set dlo[l+2]; past the capacity, raise dlo[nlo] and add none.
// 16 lanes a box: lane ci < 8 writes child ci.
__global__ void k_atree_emit(int* __restrict__ dlo, int nlo, int cap, int nscan, int l, int D,
                             const int* __restrict__ scan,
                             uint32_t* __restrict__ key, int* __restrict__ lev,
                             int* __restrict__ par, int* __restrict__ s0, int* __restrict__ s1,
                             int* __restrict__ t0, int* __restrict__ t1,
                             const uint32_t* __restrict__ skey, const uint32_t* __restrict__ tkey,
                             const int* __restrict__ leaf, int* __restrict__ child) {
  const int b0 = dlo[l], b1 = dlo[l + 1], total = scan[nscan];
  const bool over = (int64_t)b1 + total > cap;
  if (blockIdx.x == 0 && threadIdx.x == 0) {  // read by the next level's kernels only
    dlo[l + 2] = over ? b1 : b1 + total;
    if (over) dlo[nlo] = 1;
  }
  const int b = b0 + (int)((blockIdx.x * blockDim.x + threadIdx.x) / kBoxLanes);
  const int k = threadIdx.x & (kBoxLanes - 1);
  const bool live = !over && b < b1 && !leaf[b];
  int bs0 = 0, bs1 = 0, bt0 = 0, bt1 = 0;
  uint32_t bkey = 0;
  if (live) bs0 = s0[b], bs1 = s1[b], bt0 = t0[b], bt1 = t1[b], bkey = key[b];
  int sb[9], tb[9];
  child_bounds_group(skey, tkey, live, bkey, l, D, bs0, bs1, bt0, bt1, sb, tb);
  if (!live || k >= 8) return;
  const int ci = k;
  if (sb[ci + 1] == sb[ci] && tb[ci + 1] == tb[ci]) return;
  int pos = b1 + scan[b - b0];
  for (int cj = 0; cj < ci; ++cj) pos += (sb[cj + 1] > sb[cj] || tb[cj + 1] > tb[cj]) ? 1 : 0;
  key[pos] = (bkey << 3) | (uint32_t)ci;
  lev[pos] = l + 1;
  par[pos] = b;
  s0[pos] = sb[ci];
  s1[pos] = sb[ci + 1];
  t0[pos] = tb[ci];
  t1[pos] = tb[ci + 1];
  child[8 * b + ci] = pos;
}

unsigned nblocks(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// exclusive scan of in[0..n) into out[0..n], out[n] = total
cudaError_t scan_ints(const int* in, int* out, int64_t n, int* sums, cudaStream_t st,
                      int* nl) {
  const unsigned nb = nblocks(n, 1024);
  k_scan_chunks<<<nb, 1024, 0, st>>>(in, out, n, sums);
  k_scan_top<<<1, 1024, 0, st>>>(sums, (int)nb);
  k_scan_add<<<nb, 1024, 0, st>>>(out, n, sums, out + n, in + n - 1);
  *nl += 3;
  return cudaGetLastError();
}

// sort one point set into leaf order; fills start[], the SoA copies and perm
template <int D>
cudaError_t sort_points(const fmm_plan_s* P, const Workspace& ws, int64_t n, const double* x,
                        const double* w, int* start, double* const* ox, double* ow, int* perm,
                        float4* rel, cudaStream_t st, int* nl) {
  const int L = P->desc.levels;
  const int64_t nleaf = nbox_at(D, L);
  cudaMemsetAsync(ws.counts, 0, sizeof(int) * nleaf, st);
  if (n == 0) {
    cudaMemsetAsync(start, 0, sizeof(int) * (nleaf + 1), st);
    return cudaGetLastError();
  }
  k_bin<D><<<nblocks(n, 256), 256, 0, st>>>(n, x, ws.geom, L, ws.keys_a, ws.vals_a, ws.counts,
                                            ws.geom);
  ++*nl;
  cudaError_t e = scan_ints(ws.counts, start, nleaf, ws.hist_sums, st, nl);
  if (e != cudaSuccess) return e;
  const int bits = D * L;
  const int nblk = (int)nblocks(n, kRsBlock);
  uint32_t* ka = ws.keys_a;
  uint32_t* kb = ws.keys_b;
  int* va = ws.vals_a;
  int* vb = ws.vals_b;
  for (int shift = 0; shift < bits; shift += 8) {
    k_rs_hist<<<nblk, kRsBlock, 0, st>>>(ka, (int)n, shift, ws.hist, nblk);
    ++*nl;
    const int64_t nh = 256LL * nblk;
    const unsigned nb = nblocks(nh, 1024);
    k_scan_chunks<<<nb, 1024, 0, st>>>(ws.hist, ws.hist, nh, ws.hist_sums);
    k_scan_top<<<1, 1024, 0, st>>>(ws.hist_sums, (int)nb);
    k_scan_add<<<nb, 1024, 0, st>>>(ws.hist, nh, ws.hist_sums, nullptr, nullptr);
    k_rs_scatter<<<nblk, kRsBlock, 0, st>>>(ka, va, kb, vb, (int)n, shift, ws.hist, nblk);
    *nl += 4;
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (rel)
    k_gather_rel<<<nblocks(n, 256), 256, 0, st>>>((int)n, va, ka, x, w, ws.geom, P->desc.levels,
                                                  rel, perm);
  else
    k_gather<D><<<nblocks(n, 256), 256, 0, st>>>((int)n, va, x, w, ox[0], ox[1],
                                                 D == 3 ? ox[2] : ox[0], ow, perm);
  ++*nl;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_set_geom(const fmm_plan_s* P, const Workspace& ws, int64_t n_src,
                            const double* src, int64_t n_tgt, const double* tgt,
                            cudaStream_t st, int* nl) {
  const fmm_plan_desc& d = P->desc;
  const int depth = d.levels > 0 ? d.levels : -d.levels;  // adaptive: deepest level
  if (d.root_size > 0.0) {
    k_geom_fixed<<<1, 1, 0, st>>>(ws.geom, d.root_lo[0], d.root_lo[1], d.d == 3 ? d.root_lo[2] : 0.0,
                                  d.root_size, depth);
    ++*nl;
    return cudaGetLastError();
  }
  const int nb = ws.nbbox_blocks;
  if (P->pd.d == 3) {
    k_bbox_partial<3><<<nb, 256, 0, st>>>(n_src, src, n_tgt, tgt, ws.bbox);
    k_bbox_final<3><<<1, 32, 0, st>>>(nb, ws.bbox, ws.geom, depth);
  } else {
    k_bbox_partial<2><<<nb, 256, 0, st>>>(n_src, src, n_tgt, tgt, ws.bbox);
    k_bbox_final<2><<<1, 32, 0, st>>>(nb, ws.bbox, ws.geom, depth);
  }
  *nl += 2;
  return cudaGetLastError();
}

cudaError_t launch_build_tree(const fmm_plan_s* P, const Workspace& ws, int64_t n_src,
                              const double* src, const double* w, int64_t n_tgt,
                              const double* tgt, cudaStream_t st, int* nl) {
  cudaError_t e;
  const bool shared = ws.tstart == ws.sstart;  // targets are the sources: sorted once
  if (P->pd.d == 3) {
    // the FP32 path keeps only the box-relative float4 copies
    e = sort_points<3>(P, ws, n_src, src, w, ws.sstart, ws.sx, ws.sw, ws.sperm, ws.sxr, st, nl);
    if (e != cudaSuccess || shared) return e;
    e = sort_points<3>(P, ws, n_tgt, tgt, nullptr, ws.tstart, ws.tx, nullptr, ws.tperm, ws.txr,
                       st, nl);
  } else {
    e = sort_points<2>(P, ws, n_src, src, w, ws.sstart, ws.sx, ws.sw, ws.sperm, nullptr, st, nl);
    if (e != cudaSuccess || shared) return e;
    e = sort_points<2>(P, ws, n_tgt, tgt, nullptr, ws.tstart, ws.tx, nullptr, ws.tperm, nullptr,
                       st, nl);
  }
  return e;
}

namespace {

// sort one point set by Morton code at depth D into the FP64 SoA arrays,
// keeping the sorted codes
cudaError_t asort_points(const Workspace& ws, int64_t n, const double* x, const double* w,
                         double* const* ox, double* ow, int* perm, uint32_t* okey, int D,
                         cudaStream_t st, int* nl) {
  if (n == 0) return cudaGetLastError();
  k_amorton<<<nblocks(n, 256), 256, 0, st>>>(n, x, ws.geom, D, ws.keys_a, ws.vals_a, ws.geom);
  ++*nl;
  const int bits = 3 * D;
  const int nblk = (int)nblocks(n, kRsBlock);
  uint32_t* ka = ws.keys_a;
  uint32_t* kb = ws.keys_b;
  int* va = ws.vals_a;
  int* vb = ws.vals_b;
  for (int shift = 0; shift < bits; shift += 8) {
    k_rs_hist<<<nblk, kRsBlock, 0, st>>>(ka, (int)n, shift, ws.hist, nblk);
    const int64_t nh = 256LL * nblk;
    const unsigned nb = nblocks(nh, 1024);
    k_scan_chunks<<<nb, 1024, 0, st>>>(ws.hist, ws.hist, nh, ws.hist_sums);
    k_scan_top<<<1, 1024, 0, st>>>(ws.hist_sums, (int)nb);
    k_scan_add<<<nb, 1024, 0, st>>>(ws.hist, nh, ws.hist_sums, nullptr, nullptr);
    k_rs_scatter<<<nblk, kRsBlock, 0, st>>>(ka, va, kb, vb, (int)n, shift, ws.hist, nblk);
    *nl += 5;
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  cudaMemcpyAsync(okey, ka, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st);
  k_gather<3><<<nblocks(n, 256), 256, 0, st>>>((int)n, va, x, w, ox[0], ox[1], ox[2], ow, perm);
  ++*nl;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_build_adaptive(const fmm_plan_s* P, const Workspace& ws, int64_t n_src,
                                  const double* src, const double* w, int64_t n_tgt,
                                  const double* tgt, cudaStream_t st, int* nl, ATree* t,
                                  int* overflow) {
  const int D = -P->desc.levels;
  *overflow = 0;
  cudaError_t e = asort_points(ws, n_src, src, w, ws.sx, ws.sw, ws.sperm, ws.skey, D, st, nl);
  if (e != cudaSuccess) return e;
  if (ws.asxh && n_src > 0) {  // the float leaf pass's split copy of the sorted sources
    k_split_points<<<nblocks(n_src, 256), 256, 0, st>>>(n_src, ws.sx[0], ws.sx[1], ws.sx[2],
                                                        ws.sw, ws.asxh, ws.asxl);
    ++*nl;
  }
  if (ws.tkey != ws.skey) {  // else the targets are the sources, sorted once
    e = asort_points(ws, n_tgt, tgt, nullptr, ws.tx, nullptr, ws.tperm, ws.tkey, D, st, nl);
    if (e != cudaSuccess) return e;
  }
  // Level by level without the host: the level offsets live on the device
  // (dlo[0..D+2], overflow flag at dlo[D+3]) and every level's kernels read
  // their box range there.  One read at the end.  The host sizes each
  // level's launches by a bound on its box count: level l+1 holds at most 8
  // children of each split box of level l, there are at most n / (max_leaf + 1)
  // split boxes (their point sets are disjoint), and no box is empty.
  const int nlo = D + 3;
  int* dlo = ws.aloff;
  const int cap = (int)ws.anb_cap;
  const int64_t npts = n_src + (ws.tkey != ws.skey ? n_tgt : 0);
  const int64_t splits_cap = (n_src + n_tgt) / ((int64_t)P->desc.max_leaf + 1);
  k_atree_root<<<1, 1, 0, st>>>(ws.alev, ws.apar, ws.akey, ws.as0, ws.as1, ws.at0, ws.at1,
                                (int)n_src, (int)n_tgt, dlo, nlo);
  ++*nl;
  int64_t bound = 1;  // boxes of level l at most
  for (int l = 0; l <= D; ++l) {
    // (at least one thread and count: a level past the last split holds no
    // box, and its emit still has to carry the offset down)
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(bound, cap));
    // counts past the level's boxes stay zero, so the scan of nb counts ends
    // in the level's total
    cudaMemsetAsync(ws.anch, 0, sizeof(int) * (size_t)nb, st);
    k_atree_split<<<nblocks((int64_t)nb * kBoxLanes, 256), 256, 0, st>>>(
        dlo, l, D, P->desc.max_leaf, ws.akey, ws.as0, ws.as1, ws.at0, ws.at1, ws.skey, ws.tkey,
        ws.aleaf, ws.achild, ws.anch);
    ++*nl;
    if (l == D) break;
    e = scan_ints(ws.anch, ws.ascan, nb, ws.hist_sums, st, nl);
    if (e != cudaSuccess) return e;
    k_atree_emit<<<nblocks((int64_t)nb * kBoxLanes, 256), 256, 0, st>>>(
        dlo, nlo, cap, nb, l, D, ws.ascan, ws.akey, ws.alev, ws.apar, ws.as0, ws.as1, ws.at0,
        ws.at1, ws.skey, ws.tkey, ws.aleaf, ws.achild);
    ++*nl;
    bound = std::min<int64_t>(8 * std::min<int64_t>(bound, splits_cap), std::max<int64_t>(npts, 1));
  }
  // the levels' coordinate bounds (for the adaptive M2L's windows), read in the same copy
  int* dbnd = dlo + nlo + 1;
  const int nbnd = 6 * (D + 2);
  k_abounds_init<<<1, 128, 0, st>>>(dbnd, nbnd);
  k_abounds<<<nblocks(cap, 256), 256, 0, st>>>(dlo, D, ws.alev, ws.akey, dbnd);
  *nl += 2;
  static_assert(sizeof(P->abnd) >= sizeof(int) * 6 * (FMM_MAX_ADEPTH + 2), "level bounds");
  int hlo[FMM_MAX_ADEPTH + 4 + 6 * (FMM_MAX_ADEPTH + 2)];
  cudaMemcpyAsync(hlo, dlo, sizeof(int) * (nlo + 1 + nbnd), cudaMemcpyDeviceToHost, st);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  std::copy(hlo + nlo + 1, hlo + nlo + 1 + nbnd, const_cast<fmm_plan_s*>(P)->abnd);
  if (hlo[nlo]) {
    *overflow = 1;
    return cudaSuccess;
  }
  int loff[FMM_MAX_ADEPTH + 2];
  int maxlev = 0;
  for (int l = 0; l <= D + 1; ++l) loff[l] = hlo[l];
  for (int l = 1; l <= D; ++l)
    if (hlo[l + 1] > hlo[l]) maxlev = l;
  t->key = ws.akey;
  t->lev = ws.alev;
  t->par = ws.apar;
  t->child = ws.achild;
  t->s0 = ws.as0;
  t->s1 = ws.as1;
  t->t0 = ws.at0;
  t->t1 = ws.at1;
  t->leaf = ws.aleaf;
  for (int l = 0; l <= FMM_MAX_ADEPTH + 1; ++l) t->loff[l] = l <= maxlev + 1 ? loff[l] : loff[maxlev + 1];
  t->maxlev = maxlev;
  // dense index of levels 0..glev (one load per lookup there)
  const int glev = std::min(maxlev, FMM_AGRID_LEVELS);
  const int nbox = loff[maxlev + 1];
  cudaMemsetAsync(ws.agrid, 0xff, sizeof(int) * (size_t)agrid_offset(glev + 1), st);
  k_agrid_fill<<<nblocks(nbox, 256), 256, 0, st>>>(nbox, glev, ws.akey, ws.alev, ws.agrid);
  ++*nl;
  t->grid = ws.agrid;
  t->grid_levels = glev;
  return cudaGetLastError();
}
