// Adaptive trees in the mixed-precision modes: the leaf pass, one warp per
// leaf (3D; the FP64 form keeps the block-per-leaf kernel of leaf.cu).
//
//  * k_aleaf_w: L2P from the leaf's local expansion (nested Horner), and P2P
//    over the U list, the W boxes of at most |j| sources and the X pairs of
//    the leaf's ancestors holding at most |j| targets (the lists of the
//    classical adaptive FMM with the direct-sum rule for small boxes).  The
//    27-neighbour scans run one lookup per lane and walk the hits from a
//    ballot, so the dependent lookups of a scan overlap.  A source chunk of 32
//    is staged in shared memory box-relative; the leaf's targets are spread
//    over the lanes with gs = 32 / (targets rounded up to a power of two)
//    lanes per target, each taking every gs-th source, the groups summed by
//    shuffles at the end.  The kernel needs no per-thread recurrence scratch,
//    so four leaves share a block at full occupancy.
//  * k_am2p_w: the W boxes holding more than |j| sources (M2P, the float
//    derivative recurrence per target), only for the leaves k_aleaf_w flagged;
//    each warp adds them to its own targets' potentials.
#include "adaptive.cuh"
#include "expansions.cuh"

namespace {

constexpr int kLW = 4;  // leaves (warps) per block of k_aleaf_w
constexpr int kLStack = 8 * (FMM_MAX_ADEPTH + 1);

__device__ __forceinline__ float rsqrt_hw(float x) {  // hardware approximation, ~2^-23
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// the far field at box-relative u: nested Horner over the decompressed
// Lt_m / m! (full layout: m_0 within rows, m_1 over rows, m_s over slabs)
__device__ float far_horner(const PlanDev& pd, const float* __restrict__ cb, float u0, float u1,
                            float u2) {
  const int p = pd.p;
  float F = 0.f;
  for (int ms = p; ms >= 0; --ms) {
    float S = 0.f;
    for (int m1 = p - ms; m1 >= 0; --m1) {
      const int base = pd.frow[ms * (p + 1) + m1], len = p - ms - m1 + 1;
      float v = cb[base + len - 1];
      for (int k = len - 2; k >= 0; --k) v = fmaf(v, u0, cb[base + k]);
      S = fmaf(S, u1, v);
    }
    F = fmaf(F, u2, S);
  }
  return F;
}

// (x - c) / s from float pairs x = xh + xl, c = ch + cl, inv_s a power of two
__device__ __forceinline__ float box_rel(float xh, float xl, float ch, float cl, float inv_s) {
  return __fmul_rn(__fadd_rn(__fsub_rn(xh, ch), __fsub_rn(xl, cl)), inv_s);
}

// neighbour k (0..26) of coordinates c
__device__ __forceinline__ void nbr(const int* c, int k, int* nc) {
  nc[0] = c[0] + k % 3 - 1;
  nc[1] = c[1] + (k / 3) % 3 - 1;
  nc[2] = c[2] + k / 9 - 1;
}

// calls f(A) for every lane's box A whose predicate holds, in lane order
// (warp-uniform: every lane calls f with the same A)
template <typename F>
__device__ __forceinline__ void for_hits(bool pred, int A, F&& f) {
  unsigned m = __ballot_sync(0xffffffffu, pred);
  while (m) {
    const int k = __ffs(m) - 1;
    m &= m - 1;
    f(__shfl_sync(0xffffffffu, A, k));
  }
}

__global__ void __launch_bounds__(32 * kLW) k_aleaf_w(
    PlanDev pd, const Geom* __restrict__ g, ATree t, const double* __restrict__ lc,
    const double* __restrict__ tx0, const double* __restrict__ tx1,
    const double* __restrict__ tx2, const int* __restrict__ tperm, const float4* __restrict__ sxh,
    const float4* __restrict__ sxl, double* __restrict__ phi, unsigned char* __restrict__ need_m2p,
    int* __restrict__ err) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.x * kLW + warp;
  if (b >= t.loff[t.maxlev + 1] || !t.leaf[b] || t.t1[b] == t.t0[b]) return;  // warp-uniform
  const int nfull = pd.nfull, nj = pd.nj;
  int l, bc[3];
  abox(t, b, &l, bc);
  double cb[3], s;
  abox_center(g, l, bc, cb, &s);
  const double inv_s = 1.0 / s;
  // the centre as float pairs, so that a source's box-relative coordinate
  // ((xh - ch) + (xl - cl)) / s comes out of float arithmetic to a few
  // float roundings of itself (s is a power of two)
  const float ch[3] = {(float)cb[0], (float)cb[1], (float)cb[2]};
  const float cl[3] = {(float)(cb[0] - (double)ch[0]), (float)(cb[1] - (double)ch[1]),
                       (float)(cb[2] - (double)ch[2])};
  const float inv_sf = (float)inv_s;
  extern __shared__ __align__(16) float smw[];
  const int per_warp = ((nfull + 3) & ~3) + 4 * 32;
  float* a = smw + (size_t)warp * per_warp;                      // decompressed Lt / m!
  float4* stage = reinterpret_cast<float4*>(a + ((nfull + 3) & ~3));  // 32 staged sources
  const bool has_local = l >= 2;
  if (has_local) {
    for (int q = lane; q < nj; q += 32) a[q] = (float)lc[(size_t)b * nj + q];
    __syncwarp();
    decompress_warp<float>(pd, a, s, lane);
    for (int q = lane; q < nfull; q += 32) a[q] *= pd.inv_fact_f[q];
    __syncwarp();
  }
  const int kern = pd.kernel;
  const float nl2e = -(float)(pd.lam * s) * 1.4426950408889634f;
  double near_scale;  // box units -> physical
  if (kern == FMM_KERNEL_LAPLACE) near_scale = inv_s * (1.0 / (4.0 * 3.14159265358979323846));
  else if (kern == FMM_KERNEL_YUKAWA) near_scale = inv_s;
  else near_scale = s;
  const int t0 = t.t0[b], t1 = t.t1[b];
  bool flag = false;  // a W box of more than |j| sources: M2P in k_am2p_w
  for (int tb = t0; tb < t1; tb += 64) {  // superblocks of 64 targets (one below max_leaf 64)
    const int nt = min(64, t1 - tb);
    const int nblk = nt > 32 ? 2 : 1;
    int gs = 1;
    if (nt <= 32) {
      int tp = 1;
      while (tp < nt) tp <<= 1;
      gs = 32 / tp;
    }
    const int sub = lane & (gs - 1);
    int ti[2];
    bool val[2];
    float u[2][3];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      ti[k] = tb + k * 32 + lane / gs;
      val[k] = k < nblk && ti[k] < tb + nt;
      u[k][0] = u[k][1] = u[k][2] = 0.f;
      if (val[k]) {  // the sources' arithmetic: a point that is both gets equal coordinates
        const double x[3] = {tx0[ti[k]], tx1[ti[k]], tx2[ti[k]]};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const float h = (float)x[d], o = (float)(x[d] - (double)h);
          u[k][d] = box_rel(h, o, ch[d], cl[d], inv_sf);
        }
      }
    }
    float near[2] = {0.f, 0.f};
    // P2P against the sources of box A (own leaf: x == y skipped)
    auto p2p = [&](int A) {
      const bool own = A == b;
      const int s0 = t.s0[A], s1 = t.s1[A];
      for (int jb = s0; jb < s1; jb += 32) {
        const int n = min(32, s1 - jb);
        __syncwarp();
        if (lane < n) {
          const float4 h = sxh[jb + lane], o = sxl[jb + lane];
          stage[lane] = make_float4(box_rel(h.x, o.x, ch[0], cl[0], inv_sf),
                                    box_rel(h.y, o.y, ch[1], cl[1], inv_sf),
                                    box_rel(h.z, o.z, ch[2], cl[2], inv_sf), h.w);
        }
        __syncwarp();
        for (int q = sub; q < n; q += gs) {
          const float4 v = stage[q];
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            if (k < nblk) {
              const float dx = u[k][0] - v.x, dy = u[k][1] - v.y, dz = u[k][2] - v.z;
              const float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, own ? 0.f : 1e-30f)));
              const float ri = rsqrt_hw(r2);
              float gv;
              if (kern == FMM_KERNEL_LAPLACE) {
                gv = ri;
              } else if (kern == FMM_KERNEL_YUKAWA) {
                float e;
                asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(nl2e * r2 * ri));
                gv = e * ri;
              } else {
                gv = r2 * ri;
              }
              if (own && r2 == 0.f) gv = 0.f;
              near[k] = fmaf(v.w, gv, near[k]);
            }
          }
        }
      }
    };
    // U: coarser adjacent leaves (neighbours of each ancestor at its level)
    for (int lp = l - 1; lp >= 0; --lp) {
      const int an[3] = {bc[0] >> (l - lp), bc[1] >> (l - lp), bc[2] >> (l - lp)};
      int A = -1;
      bool hit = false;
      if (lane < 27) {
        int nc[3];
        nbr(an, lane, nc);
        A = alookup(t, lp, nc);
        hit = A >= 0 && t.leaf[A] && aadjacent(lp, nc, l, bc);
      }
      for_hits(hit, A, p2p);
    }
    // colleagues: leaves -> U (the leaf itself among them); the others'
    // descendants: adjacent leaves -> U, non-adjacent boxes -> W
    {
      int C = -1;
      if (lane < 27) {
        int nc[3];
        nbr(bc, lane, nc);
        C = alookup(t, l, nc);
      }
      const bool isleaf = C >= 0 && t.leaf[C];
      for_hits(isleaf, C, p2p);
      for_hits(C >= 0 && !isleaf, C, [&](int Cn) {
        int stack[kLStack];
        int sp = 0;
        for (int ci = 0; ci < 8; ++ci)
          if (t.child[8 * Cn + ci] >= 0) stack[sp++] = t.child[8 * Cn + ci];
        while (sp > 0) {
          const int E = stack[--sp];
          int le, ce[3];
          abox(t, E, &le, ce);
          if (!aadjacent(le, ce, l, bc)) {
            if (t.s1[E] - t.s0[E] <= nj) p2p(E);  // W box of at most |j| sources
            else flag = true;
          } else if (t.leaf[E]) {
            p2p(E);
          } else {
            for (int ci = 0; ci < 8; ++ci) {
              const int F = t.child[8 * E + ci];
              if (F < 0) continue;
              if (sp < kLStack) stack[sp++] = F;
              else if (lane == 0) atomicOr(err, 4);  // cannot happen: 7 siblings per level
            }
          }
        }
      });
    }
    // X pairs of the leaf and its ancestors C (level >= 2) holding at most
    // |j| targets: the leaves coarser than C, adjacent to C's parent but not
    // to C, found among the neighbours of C's ancestors
    {
      int lc_ = l;
      for (int Cb = b; Cb >= 0 && lc_ >= 2 && t.t1[Cb] - t.t0[Cb] <= nj; Cb = t.par[Cb], --lc_) {
        const int cc[3] = {bc[0] >> (l - lc_), bc[1] >> (l - lc_), bc[2] >> (l - lc_)};
        const int pc[3] = {cc[0] >> 1, cc[1] >> 1, cc[2] >> 1};
        for (int lp = lc_ - 1; lp >= 0; --lp) {
          const int an[3] = {cc[0] >> (lc_ - lp), cc[1] >> (lc_ - lp), cc[2] >> (lc_ - lp)};
          int A = -1;
          bool hit = false;
          if (lane < 27) {
            int nc[3];
            nbr(an, lane, nc);
            A = alookup(t, lp, nc);
            hit = A >= 0 && t.leaf[A] && aadjacent(lp, nc, lc_ - 1, pc) &&
                  !aadjacent(lp, nc, lc_, cc);
          }
          for_hits(hit, A, p2p);
        }
      }
    }
    // the groups' partial sums, then far + near
#pragma unroll
    for (int k = 0; k < 2; ++k)
      for (int off = gs >> 1; off > 0; off >>= 1)
        near[k] += __shfl_xor_sync(0xffffffffu, near[k], off);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (sub == 0 && val[k]) {
        const float far = has_local ? far_horner(pd, a, u[k][0], u[k][1], u[k][2]) : 0.f;
        phi[tperm[ti[k]]] = (double)far + near_scale * (double)near[k];
      }
    }
  }
  if (lane == 0) need_m2p[b] = flag ? 1 : 0;
}

// M2P over the W boxes of more than |j| sources, for the flagged leaves: one
// warp per leaf, lane k owning targets k and k + 32 of each 64-target block;
// the box's multipole staged in shared memory, the float derivative
// recurrence per target with its two-degree slices in shared memory.
__global__ void __launch_bounds__(32) k_am2p_w(PlanDev pd, const Geom* __restrict__ g, ATree t,
                                               const double* __restrict__ mp,
                                               const double* __restrict__ tx0,
                                               const double* __restrict__ tx1,
                                               const double* __restrict__ tx2,
                                               const int* __restrict__ tperm,
                                               const unsigned char* __restrict__ need_m2p,
                                               double* __restrict__ phi, int* __restrict__ err) {
  const int b = blockIdx.x, lane = threadIdx.x;
  if (b >= t.loff[t.maxlev + 1] || !t.leaf[b] || t.t1[b] == t.t0[b] || !need_m2p[b]) return;
  const int nj = pd.nj, p = pd.p;
  int l, bc[3];
  abox(t, b, &l, bc);
  double cb[3], s;
  abox_center(g, l, bc, cb, &s);
  const double inv_s = 1.0 / s;
  extern __shared__ __align__(16) float smm[];
  float* bt = smm;  // the W box's multipole
  const int sl = min(pd.c, p + 1) * (p + 1);
  const int per = (kernel_screened(pd.kernel) ? 6 : 3) * sl;
  float* S = smm + ((nj + 3) & ~3) + lane * per;
  const int t0 = t.t0[b], t1 = t.t1[b];
  for (int tb = t0; tb < t1; tb += 64) {
    int ti[2];
    bool val[2];
    float u[2][3];
    float acc[2] = {0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      ti[k] = tb + k * 32 + lane;
      val[k] = ti[k] < t1;
      u[k][0] = u[k][1] = u[k][2] = 0.f;
      if (val[k]) {
        u[k][0] = (float)((tx0[ti[k]] - cb[0]) * inv_s);
        u[k][1] = (float)((tx1[ti[k]] - cb[1]) * inv_s);
        u[k][2] = (float)((tx2[ti[k]] - cb[2]) * inv_s);
      }
    }
    auto m2p = [&](int E, int le, const int* ce) {
      double c2[3], s2;
      abox_center(g, le, ce, c2, &s2);
      __syncwarp();
      for (int q = lane; q < nj; q += 32) bt[q] = (float)mp[(size_t)E * nj + q];
      __syncwarp();
      const double is2 = 1.0 / s2;
      const float ratio = (float)(s * is2);  // a power of two
      const float off[3] = {(float)((cb[0] - c2[0]) * is2), (float)((cb[1] - c2[1]) * is2),
                            (float)((cb[2] - c2[2]) * is2)};
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        if (!val[k]) continue;
        const float y[3] = {fmaf(u[k][0], ratio, off[0]), fmaf(u[k][1], ratio, off[1]),
                            fmaf(u[k][2], ratio, off[2])};
        float v = 0.f;
        deriv_point<float>(pd, y, (float)(pd.lam * s2), (float)deriv_scale(pd, s2), S, sl,
                           [&](int pos, float h) { v = fmaf(h, bt[pos], v); });
        acc[k] += v;
      }
    };
    int C = -1;
    if (lane < 27) {
      int nc[3];
      nbr(bc, lane, nc);
      C = alookup(t, l, nc);
    }
    for_hits(C >= 0 && !t.leaf[C], C, [&](int Cn) {
      int stack[kLStack];
      int sp = 0;
      for (int ci = 0; ci < 8; ++ci)
        if (t.child[8 * Cn + ci] >= 0) stack[sp++] = t.child[8 * Cn + ci];
      while (sp > 0) {
        const int E = stack[--sp];
        int le, ce[3];
        abox(t, E, &le, ce);
        if (!aadjacent(le, ce, l, bc)) {
          if (t.s1[E] - t.s0[E] > nj) m2p(E, le, ce);
        } else if (!t.leaf[E]) {
          for (int ci = 0; ci < 8; ++ci) {
            const int F = t.child[8 * E + ci];
            if (F < 0) continue;
            if (sp < kLStack) stack[sp++] = F;
            else if (lane == 0) atomicOr(err, 4);
          }
        }
      }
    });
#pragma unroll
    for (int k = 0; k < 2; ++k)
      if (val[k]) phi[tperm[ti[k]]] += (double)acc[k];  // each target in one warp: no race
  }
}

}  // namespace

// the leaf pass of a 3D adaptive tree in float (mixed-precision plans)
cudaError_t launch_adaptive_leaf_warp(const fmm_plan_s* P, const Workspace& ws, const ATree& t,
                                      double* phi, cudaStream_t st, int* nl) {
  const PlanDev& pd = P->pd;
  const int nbox = t.loff[t.maxlev + 1];
  const size_t sm1 = sizeof(float) * kLW * (size_t)(((pd.nfull + 3) & ~3) + 4 * 32);
  cudaFuncSetAttribute(k_aleaf_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
  k_aleaf_w<<<(unsigned)((nbox + kLW - 1) / kLW), 32 * kLW, sm1, st>>>(
      pd, ws.geom, t, ws.lc, ws.tx[0], ws.tx[1], ws.tx[2], ws.tperm, ws.asxh, ws.asxl, phi,
      ws.am2p, &ws.geom->flag);
  const int sl = std::min(pd.c, pd.p + 1) * (pd.p + 1);
  const int per = (kernel_screened(pd.kernel) ? 6 : 3) * sl;
  const size_t sm2 = sizeof(float) * ((size_t)((pd.nj + 3) & ~3) + (size_t)32 * per);
  cudaFuncSetAttribute(k_am2p_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
  k_am2p_w<<<(unsigned)nbox, 32, sm2, st>>>(pd, ws.geom, t, ws.mp, ws.tx[0], ws.tx[1], ws.tx[2],
                                            ws.tperm, ws.am2p, phi, &ws.geom->flag);
  *nl += 2;
  return cudaGetLastError();
}
