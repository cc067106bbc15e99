// Leaf evaluation: L2P (Sec. 3.3) and the P2P near field (eq. (1) over the 3^d
// adjacent leaves), fused in one kernel, one block per target leaf box.
//
// Coordinates are taken relative to the target box centre in units of its
// side s (u = (x - c)/s), so the far field is sum_m (Dt_m / m!) u^m with
// Dt = M Lt (box-scaled derivatives) and the near field uses u_t - u_s.
// A group of `tpt` threads shares one target: the lanes split the polynomial
// rows and the source list, then reduce with warp shuffles.  The result is
// written straight to the caller's order through the target permutation.
#include <algorithm>

#include "adaptive.cuh"
#include "expansions.cuh"
#include "f32x2.cuh"
#include "passes_f32.cuh"

namespace {

constexpr int kThreads = 128;

template <typename K>
void set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double exp_t(double x) { return exp(x); }
__device__ __forceinline__ float exp_t(float x) { return __expf(x); }
__device__ __forceinline__ double log_t(double x) { return log(x); }
__device__ __forceinline__ float log_t(float x) { return __logf(x); }
__device__ __forceinline__ void sincos_t(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ void sincos_t(float x, float* s, float* c) { sincosf(x, s, c); }

// Near-field pair in box units: r2 = |u_t - u_s|^2 > 0.  Adds to the running
// potential sum `v` (scaled later by kPhiScale) and gradient factor `f1`
// (grad G = (u_t - u_s) * f1, scaled later by kGradScale).
template <int K, int D, typename T>
__device__ __forceinline__ void pair_kernel(T r2, T lam, T& v, T& f1) {
  if (K == FMM_KERNEL_LAPLACE && D == 3) {
    const T ri = rsqrt_t(r2);
    v = ri;
    f1 = -ri * ri * ri;
  } else if (K == FMM_KERNEL_LAPLACE && D == 2) {
    v = (T)0.5 * log_t(r2);
    f1 = (T)1 / r2;
  } else if (K == FMM_KERNEL_BIHARMONIC && D == 2) {  // r^2 log r, f1 = 2 log r + 1
    const T lg = log_t(r2);
    v = (T)0.5 * r2 * lg;
    f1 = lg + (T)1;
  } else if (K == FMM_KERNEL_YUKAWA) {
    const T ri = rsqrt_t(r2);
    const T r = r2 * ri;
    const T e = exp_t(-lam * r);
    v = e * ri;
    f1 = e * (-lam * ri * ri - ri * ri * ri);
  } else if (K == FMM_KERNEL_HELMHOLTZ || K == kHelmIm) {
    // real part cos(k r)/r: f1 = -k sin/r^2 - cos/r^3; imaginary part
    // sin(k r)/r: f1 = k cos/r^2 - sin/r^3 (lam = kappa in box units)
    const T ri = rsqrt_t(r2);
    T sn, cs;
    sincos_t(lam * (r2 * ri), &sn, &cs);
    if (K == FMM_KERNEL_HELMHOLTZ) {
      v = cs * ri;
      f1 = (-lam * sn - cs * ri) * ri * ri;
    } else {
      v = sn * ri;
      f1 = (lam * cs - sn * ri) * ri * ri;
    }
  } else {  // biharmonic 3D: G = r
    const T ri = rsqrt_t(r2);
    v = r2 * ri;
    f1 = ri;
  }
}

template <int K, int D, typename T, bool GRAD>
__global__ void __launch_bounds__(kThreads) k_leaf(
    PlanDev pd, const Geom* __restrict__ g, int L, const double* __restrict__ lc,
    const int* __restrict__ tstart, const double* __restrict__ tx0,
    const double* __restrict__ tx1, const double* __restrict__ tx2,
    const int* __restrict__ tperm, const int* __restrict__ sstart,
    const double* __restrict__ sx0, const double* __restrict__ sx1,
    const double* __restrict__ sx2, const double* __restrict__ sw, double* __restrict__ phi,
    double* __restrict__ grad) {
  const int b = blockIdx.x;
  const int t0 = tstart[b], t1 = tstart[b + 1];
  if (t0 == t1) return;
  const int p = pd.p, nfull = pd.nfull, nj = pd.nj;
  const int nl = 1 << L;
  extern __shared__ __align__(16) unsigned char smraw[];
  double* Dt = reinterpret_cast<double*>(smraw);               // nfull
  T* coef = reinterpret_cast<T*>(Dt + nfull);                  // nfull
  T* su = coef + nfull + ((nfull & 1) ? 1 : 0);                // D * kThreads staged sources
  T* swt = su + D * kThreads;                                  // kThreads weights
  int bc[3];
  double c[3], s;
  box_center<D>(g, L, b, bc, c, &s);
  const double inv_s = 1.0 / s;
  // far-field coefficients Dt/m!
  for (int q = threadIdx.x; q < nj; q += blockDim.x) Dt[q] = lc[(size_t)b * nj + q];
  __syncthreads();
  decompress_smem<double>(pd, Dt, s);
  for (int q = threadIdx.x; q < nfull; q += blockDim.x) coef[q] = (T)(Dt[q] * pd.inv_fact[q]);
  __syncthreads();

  const int nt = t1 - t0;
  int pw2 = 1;
  while (pw2 < min(nt, kThreads)) pw2 <<= 1;
  const int tpt = min(32, kThreads / pw2);
  const int grp = threadIdx.x / tpt, lane = threadIdx.x % tpt;
  const int per_pass = kThreads / tpt;
  const double* tx[3] = {tx0, tx1, tx2};
  const double* sx[3] = {sx0, sx1, sx2};
  const T lam = (T)(pd.lam * s);

  for (int tb = t0; tb < t1; tb += per_pass) {
    const int t = tb + grp;
    const bool valid = t < t1;
    T u[3] = {0, 0, 0};
    if (valid)
      for (int k = 0; k < D; ++k) u[k] = (T)((tx[k][t] - c[k]) * inv_s);
    // ---- far field: rows (m_s, m_1) of the full layout, split over lanes
    T far = 0, gf[3] = {0, 0, 0};
    if (valid) {
      int row = 0;
      T pz = 1, pzm = 0;  // u_s^{m_s}, m_s u_s^{m_s-1}
      const int us = D - 1;
      for (int ms = 0; ms <= p; ++ms) {
        if (D == 3) {
          T py = 1, pym = 0;
          for (int m1 = 0; m1 <= p - ms; ++m1, ++row) {
            if (row % tpt == lane) {
              const int base = pd.frow[ms * (p + 1) + m1];
              const int len = p - ms - m1 + 1;
              T v = coef[base + len - 1], dv = 0;
              for (int k = len - 2; k >= 0; --k) {
                dv = dv * u[0] + v;
                v = v * u[0] + coef[base + k];
              }
              far += v * py * pz;
              if (GRAD) {
                gf[0] += dv * py * pz;
                gf[1] += v * pym * pz;
                gf[2] += v * py * pzm;
              }
            }
            pym = pym * u[1] + py;
            py *= u[1];
          }
        } else {
          if (row % tpt == lane) {
            const int base = pd.frow[ms];
            const int len = p - ms + 1;
            T v = coef[base + len - 1], dv = 0;
            for (int k = len - 2; k >= 0; --k) {
              dv = dv * u[0] + v;
              v = v * u[0] + coef[base + k];
            }
            far += v * pz;
            if (GRAD) {
              gf[0] += dv * pz;
              gf[1] += v * pzm;
            }
          }
          ++row;
        }
        pzm = pzm * u[us] + pz;
        pz *= u[us];
      }
    }
    // ---- near field over the 3^(d-1) runs of x-adjacent leaves
    // wsum: sum w (2D Laplace) or sum w r^2 (2D biharmonic), and gw = sum w (u - y),
    // for the log(s) parts of the box scaling
    constexpr bool kBih2 = K == FMM_KERNEL_BIHARMONIC && D == 2;
    T nv = 0, ng[3] = {0, 0, 0}, wsum = 0, gw[3] = {0, 0, 0};
    const int nrun = D == 3 ? 9 : 3;
    for (int rr = 0; rr < nrun; ++rr) {
      const int dy = rr % 3 - 1, dz = rr / 3 - 1;
      const int by = bc[1] + dy, bz = D == 3 ? bc[2] + dz : 0;
      if (by < 0 || by >= nl || bz < 0 || bz >= nl) continue;
      const int bx0 = max(bc[0] - 1, 0), bx1 = min(bc[0] + 1, nl - 1);
      const int64_t rowb = D == 3 ? ((int64_t)bz * nl + by) * nl : (int64_t)by * nl;
      const int j0 = sstart[rowb + bx0], j1 = sstart[rowb + bx1 + 1];
      for (int jb = j0; jb < j1; jb += kThreads) {
        const int nj2 = min(kThreads, j1 - jb);
        __syncthreads();
        if (threadIdx.x < nj2) {
          const int j = jb + threadIdx.x;
          for (int k = 0; k < D; ++k) su[k * kThreads + threadIdx.x] = (T)((sx[k][j] - c[k]) * inv_s);
          swt[threadIdx.x] = (T)sw[j];
        }
        __syncthreads();
        if (valid) {
          for (int jj = lane; jj < nj2; jj += tpt) {
            T dxv[3], r2 = 0;
            for (int k = 0; k < D; ++k) {
              dxv[k] = u[k] - su[k * kThreads + jj];
              r2 += dxv[k] * dxv[k];
            }
            if (r2 > (T)0) {
              T v, f1;
              pair_kernel<K, D, T>(r2, lam, v, f1);
              const T wj = swt[jj];
              nv += wj * v;
              wsum += kBih2 ? wj * r2 : wj;
              if (GRAD) {
                const T fw = wj * f1;
                for (int k = 0; k < D; ++k) ng[k] += fw * dxv[k];
                if (kBih2)
                  for (int k = 0; k < D; ++k) gw[k] += wj * dxv[k];
              }
            }
          }
        }
      }
    }
    // ---- reduce over the lanes of the group
    for (int off = tpt >> 1; off > 0; off >>= 1) {
      far += __shfl_down_sync(0xffffffffu, far, off, tpt);
      nv += __shfl_down_sync(0xffffffffu, nv, off, tpt);
      wsum += __shfl_down_sync(0xffffffffu, wsum, off, tpt);
      if (GRAD)
        for (int k = 0; k < D; ++k) {
          gf[k] += __shfl_down_sync(0xffffffffu, gf[k], off, tpt);
          ng[k] += __shfl_down_sync(0xffffffffu, ng[k], off, tpt);
          if (kBih2) gw[k] += __shfl_down_sync(0xffffffffu, gw[k], off, tpt);
        }
    }
    if (valid && lane == 0) {
      double phi_scale, grad_scale;  // near-field units -> physical
      if (K == FMM_KERNEL_LAPLACE && D == 3) {
        phi_scale = 1.0 / (4.0 * 3.14159265358979323846 * s);
        grad_scale = phi_scale * inv_s;
      } else if (K == FMM_KERNEL_LAPLACE && D == 2) {
        phi_scale = 1.0;
        grad_scale = inv_s;
      } else if (kBih2) {
        phi_scale = s * s;
        grad_scale = s;
      } else if (kernel_screened(K)) {
        phi_scale = inv_s;
        grad_scale = inv_s * inv_s;
      } else {
        phi_scale = s;
        grad_scale = 1.0;
      }
      const int orig = tperm[t];
      double ph = (double)far + phi_scale * (double)nv;
      if (K == FMM_KERNEL_LAPLACE && D == 2) ph += log(s) * (double)wsum;
      if (kBih2) ph += s * s * log(s) * (double)wsum;
      if (phi) phi[orig] = ph;
      if (GRAD && grad)
        for (int k = 0; k < D; ++k)
          grad[(size_t)orig * D + k] = (double)gf[k] * inv_s + grad_scale * (double)ng[k] +
                                       (kBih2 ? 2.0 * s * log(s) * (double)gw[k] : 0.0);
    }
  }
}

template <int K, int D, typename T, bool GRAD>
void leaf_launch_g(const fmm_plan_s* P, const Workspace& ws, double* phi, double* grad,
                   cudaStream_t st) {
  const PlanDev& pd = P->pd;
  const int L = P->desc.levels;
  const size_t smem = sizeof(double) * pd.nfull + sizeof(T) * (pd.nfull + 1) +
                      sizeof(T) * (D + 1) * kThreads + 16;
  set_smem(k_leaf<K, D, T, GRAD>, smem);
  k_leaf<K, D, T, GRAD><<<(unsigned)nbox_at(D, L), kThreads, smem, st>>>(
      pd, ws.geom, L, ws.lc + ws.lev_off[L] * pd.nj, ws.tstart, ws.tx[0], ws.tx[1],
      D == 3 ? ws.tx[2] : ws.tx[0], ws.tperm, ws.sstart, ws.sx[0], ws.sx[1],
      D == 3 ? ws.sx[2] : ws.sx[0], ws.sw, phi, grad);
}

// ---------------------------------------------------------------------------
// FP32 leaf path (d = 3).
//
// The gather of the tree build gives every sorted point float (x - c_own)/s
// and its weight, c_own the centre of its own leaf.
// k_leaf_fast: the near field, one warp per target leaf (P2P in packed f32x2
// pairs).  k_leaf_far: the far field, two target leaves per warp (leaf
// decompression in shared memory, then L2P in packed f32x2).
// ---------------------------------------------------------------------------
constexpr int kFastWarps = 4;   // target leaves per block (one warp each)
constexpr int kStageSrc = 256;  // staged sources per warp and chunk

// Near-field pair in box units without a branch: the x == y pair (r2 == 0)
// contributes nothing.  Returns G's scaled value and d G / (r dr) factor.
__device__ __forceinline__ float rsqrt_fast(float x) {  // hardware approximation, ~2^-23
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}


// ---- packed pairs: two sources per instruction (f32x2 arithmetic) ----------
// Staged sources come in pairs: A = (x0, x1, y0, y1), B = (z0, z1, w0, w1)
// in box units relative to the target leaf; an odd count is padded with a
// far, weightless source.

// Accumulates one source pair into (acc, g) for the target u = (UX, UY, UZ)
// (each coordinate broadcast into both halves).  g collects sum w |f1| (u - y)
// with f1 = (1/r) dG/dr; pair_sign<K>() restores the sign of f1.
template <int K>
__host__ __device__ constexpr float pair_sign() {
  // the Helmholtz parts carry the sign of f1 themselves (it oscillates)
  return (K == FMM_KERNEL_BIHARMONIC || K == FMM_KERNEL_HELMHOLTZ || K == kHelmIm) ? 1.f : -1.f;
}

template <int K, bool GRAD, bool MASK>
__device__ __forceinline__ void pair2(const float4 A, const float4 B, f2_t UX, f2_t UY, f2_t UZ,
                                      f2_t LAM, f2_t NL2E, f2_t& acc, f2_t* g) {
  const f2_t dx = f2sub(UX, f2pack(A.x, A.y));
  const f2_t dy = f2sub(UY, f2pack(A.z, A.w));
  const f2_t dz = f2sub(UZ, f2pack(B.x, B.y));
  const f2_t W = f2pack(B.z, B.w);
  const f2_t eps = MASK ? 0ull : f2pack(1e-30f, 1e-30f);
  const f2_t r2 = f2fma(dz, dz, f2fma(dy, dy, f2fma(dx, dx, eps)));
  float r2l, r2h;
  f2unpack(r2, r2l, r2h);
  float ril = rsqrt_fast(r2l), rih = rsqrt_fast(r2h);
  if (MASK) {  // x == y contributes nothing
    ril = r2l > 0.f ? ril : 0.f;
    rih = r2h > 0.f ? rih : 0.f;
  }
  const f2_t ri = f2pack(ril, rih);
  f2_t v, f1 = 0ull;
  if (K == FMM_KERNEL_LAPLACE) {
    v = ri;
    if (GRAD) f1 = f2mul(f2mul(ri, ri), ri);  // |f1| = 1/r^3
  } else if (K == FMM_KERNEL_YUKAWA) {
    float al, ah, el, eh;
    f2unpack(f2mul(f2mul(r2, ri), NL2E), al, ah);  // -lam r log2(e)
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(el) : "f"(al));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(eh) : "f"(ah));
    v = f2mul(f2pack(el, eh), ri);                          // e^{-lam r} / r (0 if masked)
    if (GRAD) f1 = f2mul(v, f2fma(ri, ri, f2mul(LAM, ri)));  // |f1| = v (lam/r + 1/r^2)
  } else if (K == FMM_KERNEL_HELMHOLTZ || K == kHelmIm) {
    float kl, kh, sl, cl, sh, ch;
    f2unpack(f2mul(f2mul(r2, ri), LAM), kl, kh);  // kappa r
    sincosf(kl, &sl, &cl);
    sincosf(kh, &sh, &ch);
    const f2_t S = f2pack(sl, sh), Cc = f2pack(cl, ch);
    const f2_t ri2 = f2mul(ri, ri);
    if (K == FMM_KERNEL_HELMHOLTZ) {  // cos(k r)/r, f1 = -(k sin + cos/r)/r^2
      v = f2mul(Cc, ri);
      if (GRAD) f1 = f2mul(f2fma(LAM, S, f2mul(Cc, ri)), f2mul(ri2, f2pack(-1.f, -1.f)));
    } else {  // sin(k r)/r, f1 = (k cos - sin/r)/r^2
      v = f2mul(S, ri);
      if (GRAD) f1 = f2mul(f2fma(LAM, Cc, f2mul(S, f2mul(ri, f2pack(-1.f, -1.f)))), ri2);
    }
  } else {  // biharmonic: G = r, f1 = 1/r
    v = f2mul(r2, ri);
    if (GRAD) f1 = ri;
  }
  acc = f2fma(W, v, acc);
  if (GRAD) {
    const f2_t fw = f2mul(W, f1);
    g[0] = f2fma(fw, dx, g[0]);
    g[1] = f2fma(fw, dy, g[1]);
    g[2] = f2fma(fw, dz, g[2]);
  }
}

// One target per lane over source pairs k0, k0 + step, ... < npair.
template <int K, bool GRAD, bool MASK>
__device__ __forceinline__ void sweep2(const float4* __restrict__ pa, const float4* __restrict__ pb,
                                       int npair, int k0, int step, const float* u, float lam,
                                       float& acc_out, float* g_out) {
  const f2_t UX = f2pack(u[0], u[0]), UY = f2pack(u[1], u[1]), UZ = f2pack(u[2], u[2]);
  const f2_t LAM = f2pack(lam, lam);
  const float nl = -lam * 1.4426950408889634f;
  const f2_t NL2E = f2pack(nl, nl);
  f2_t acc0 = 0ull, acc1 = 0ull;
  f2_t g[3] = {0ull, 0ull, 0ull};
  int k = k0;
  for (; k + step < npair; k += 2 * step) {
    pair2<K, GRAD, MASK>(pa[k], pb[k], UX, UY, UZ, LAM, NL2E, acc0, g);
    pair2<K, GRAD, MASK>(pa[k + step], pb[k + step], UX, UY, UZ, LAM, NL2E, acc1, g);
  }
  if (k < npair) pair2<K, GRAD, MASK>(pa[k], pb[k], UX, UY, UZ, LAM, NL2E, acc0, g);
  float a, b, c, d;
  f2unpack(acc0, a, b);
  f2unpack(acc1, c, d);
  acc_out += (a + b) + (c + d);
  if (GRAD)
    for (int j = 0; j < 3; ++j) {
      float lo, hi;
      f2unpack(g[j], lo, hi);
      g_out[j] += pair_sign<K>() * (lo + hi);
    }
}

// far field (L2P) at box-relative u: sum_m Dt_m/m! u^m by rows of the full
// layout (Horner along m_0), with the analytic gradient
template <bool GRAD>
__device__ __forceinline__ float far_field(const PlanDev& pd, const float* __restrict__ cb,
                                           float u0, float u1, float u2, float* gf) {
  const int p = pd.p;
  float far = 0.f;
  float pz = 1.f, pzm = 0.f;
  for (int ms = 0; ms <= p; ++ms) {
    float py = 1.f, pym = 0.f;
    for (int m1 = 0; m1 <= p - ms; ++m1) {
      const int base = pd.frow[ms * (p + 1) + m1];
      const int len = p - ms - m1 + 1;
      float v = cb[base + len - 1], dv = 0.f;
      for (int k = len - 2; k >= 0; --k) {
        if (GRAD) dv = dv * u0 + v;
        v = v * u0 + cb[base + k];
      }
      far += v * py * pz;
      if (GRAD) {
        gf[0] += dv * py * pz;
        gf[1] += v * pym * pz;
        gf[2] += v * py * pzm;
      }
      pym = pym * u1 + py;
      py *= u1;
    }
    pzm = pzm * u2 + pz;
    pz *= u2;
  }
  return far;
}

// The near field (P2P) alone: phi (and grad) are overwritten with it, and
// k_leaf_far adds the far field afterwards (on the FP32 3D uniform path the
// two run on separate streams, the near field beside the upward and M2L
// passes).
template <int K, bool GRAD>
__global__ void __launch_bounds__(32 * kFastWarps) k_leaf_fast(
    PlanDev pd, const Geom* __restrict__ g, int L, int64_t nleaf, const int* __restrict__ tstart, const float4* __restrict__ txr, const int* __restrict__ tperm,
    const int* __restrict__ sstart, const float4* __restrict__ sxr, double* __restrict__ phi,
    double* __restrict__ grad) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t b = (int64_t)blockIdx.x * kFastWarps + warp;
  __shared__ float4 stage[kFastWarps][kStageSrc];  // kStageSrc/2 source pairs: A then B
  if (b >= nleaf) return;
  const int t0 = tstart[b], t1 = tstart[b + 1];
  if (t0 == t1) return;
  float4* pa = stage[warp];
  float4* pb = stage[warp] + kStageSrc / 2;
  const int nl = 1 << L;
  int bc[3];
  {
    int64_t t = b;
    for (int k = 0; k < 3; ++k) {
      bc[k] = (int)(t % nl);
      t /= nl;
    }
  }
  // leaf side and its reciprocal from the geometry record (no FP64 division)
  const double s = g->s_leaf, inv_s = g->inv_s_leaf;
  const float lam = (float)(pd.lam * s);
  double phi_scale, grad_scale;
  if (K == FMM_KERNEL_LAPLACE) {
    phi_scale = inv_s * (1.0 / (4.0 * 3.14159265358979323846));
    grad_scale = phi_scale * inv_s;
  } else if (kernel_screened(K)) {
    phi_scale = inv_s;
    grad_scale = inv_s * inv_s;
  } else {
    phi_scale = s;
    grad_scale = 1.0;
  }
  // Per block of up to 64 targets: nfull full slots (lane = target; 0, 1 or
  // 2 of them) and r <= 16 remainder targets split over lane groups of gs.
  for (int tb = t0; tb < t1; tb += 64) {
    const int m = min(64, t1 - tb);
    int nfull = m >> 5, r = m & 31;
    if (r > 16) {
      ++nfull;
      r = 0;
    }
    int rp = 1;
    while (rp < r) rp <<= 1;
    const int gs = r ? 32 / rp : 32;
    const int tr = lane / gs, sub = lane % gs;
    const bool two = nfull == 2, one = nfull >= 1;  // warp-uniform
    const int ta = tb + lane, tb2 = tb + 32 + lane, tc = tb + 32 * nfull + tr;
    const bool va = one && ta < t1, vb = two && tb2 < t1, vc = r > 0 && tr < r;
    float ua[3] = {0.f, 0.f, 0.f}, ub[3] = {0.f, 0.f, 0.f}, uc[3] = {0.f, 0.f, 0.f};
    if (va) {
      const float4 q = txr[ta];
      ua[0] = q.x;
      ua[1] = q.y;
      ua[2] = q.z;
    }
    if (vb) {
      const float4 q = txr[tb2];
      ub[0] = q.x;
      ub[1] = q.y;
      ub[2] = q.z;
    }
    if (vc) {
      const float4 q = txr[tc];
      uc[0] = q.x;
      uc[1] = q.y;
      uc[2] = q.z;
    }
    float na = 0.f, nb = 0.f, nc = 0.f;
    float ga[3] = {0.f, 0.f, 0.f}, gb[3] = {0.f, 0.f, 0.f}, gc[3] = {0.f, 0.f, 0.f};
    for (int rr = 0; rr < 9; ++rr) {
      const int dy = rr % 3 - 1, dz = rr / 3 - 1;
      const int by = bc[1] + dy, bz = bc[2] + dz;
      if (by < 0 || by >= nl || bz < 0 || bz >= nl) continue;
      const int bx0 = max(bc[0] - 1, 0), bx1 = min(bc[0] + 1, nl - 1);
      const int64_t rowb = ((int64_t)bz * nl + by) * nl;
      const int j0 = sstart[rowb + bx0], j1 = sstart[rowb + bx1 + 1];
      const int e1 = sstart[rowb + bx0 + 1], e2 = sstart[rowb + min(bx0 + 2, bx1 + 1)];
      for (int jb = j0; jb < j1; jb += kStageSrc) {
        const int n = min(kStageSrc, j1 - jb);
        const int npair = (n + 1) >> 1;
        __syncwarp();
        for (int k = lane; k < npair; k += 32) {
          float4 v[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int q = 2 * k + h;
            if (q < n) {
              const int j = jb + q;
              v[h] = sxr[j];
              const int bx = bx0 + (j >= e1) + (j >= e2);
              v[h].x += (float)(bx - bc[0]);
              v[h].y += (float)dy;
              v[h].z += (float)dz;
            } else {
              v[h] = make_float4(1e4f, 0.f, 0.f, 0.f);  // far and weightless
            }
          }
          pa[k] = make_float4(v[0].x, v[1].x, v[0].y, v[1].y);
          pb[k] = make_float4(v[0].z, v[1].z, v[0].w, v[1].w);
        }
        __syncwarp();
        const bool center = (dy == 0 && dz == 0);  // only the own leaf can hold x == y
        if (center) {
          if (one) sweep2<K, GRAD, true>(pa, pb, npair, 0, 1, ua, lam, na, ga);
          if (two) sweep2<K, GRAD, true>(pa, pb, npair, 0, 1, ub, lam, nb, gb);
          if (r) sweep2<K, GRAD, true>(pa, pb, npair, sub, gs, uc, lam, nc, gc);
        } else {
          if (one) sweep2<K, GRAD, false>(pa, pb, npair, 0, 1, ua, lam, na, ga);
          if (two) sweep2<K, GRAD, false>(pa, pb, npair, 0, 1, ub, lam, nb, gb);
          if (r) sweep2<K, GRAD, false>(pa, pb, npair, sub, gs, uc, lam, nc, gc);
        }
      }
    }
    if (r) {  // combine the remainder groups (groups are aligned runs of gs lanes)
      for (int off = gs >> 1; off > 0; off >>= 1) {
        nc += __shfl_xor_sync(0xffffffffu, nc, off);
        if (GRAD)
          for (int k = 0; k < 3; ++k) gc[k] += __shfl_xor_sync(0xffffffffu, gc[k], off);
      }
    }
    // write the slots in use, each lane its own targets
    const int nslot = nfull + (r ? 1 : 0);
    for (int slot = 0; slot < nslot; ++slot) {
      const bool split = slot == nfull;  // the remainder slot
      const bool valid = split ? (vc && sub == 0) : (slot == 0 ? va : vb);
      if (valid) {
        // select values, not pointers, so the per-slot arrays stay in registers
        const int t = split ? tc : (slot == 0 ? ta : tb2);
        const int orig = tperm[t];
        const float nv = split ? nc : (slot == 0 ? na : nb);
        if (phi) phi[orig] = phi_scale * (double)nv;
        if (GRAD && grad) {
          const float g0 = split ? gc[0] : (slot == 0 ? ga[0] : gb[0]);
          const float g1 = split ? gc[1] : (slot == 0 ? ga[1] : gb[1]);
          const float g2 = split ? gc[2] : (slot == 0 ? ga[2] : gb[2]);
          grad[(size_t)orig * 3 + 0] = grad_scale * (double)g0;
          grad[(size_t)orig * 3 + 1] = grad_scale * (double)g1;
          grad[(size_t)orig * 3 + 2] = grad_scale * (double)g2;
        }
      }
    }
  }
}

// far_field for two targets at once in packed f32x2 arithmetic (both halves
// share the coefficients); row bases follow the full layout: rows (ms, m1) in
// order, m0 contiguous.
template <bool GRAD>
__device__ __forceinline__ f2_t far_field2(const PlanDev& pd, const float* __restrict__ cb,
                                           f2_t U0, f2_t U1, f2_t U2, f2_t* gf) {
  const int p = pd.p;
  const f2_t one = f2pack(1.f, 1.f);
  f2_t far = 0ull, pz = one, pzm = 0ull;
  int base = 0;
  for (int ms = 0; ms <= p; ++ms) {
    f2_t py = one, pym = 0ull;
    for (int m1 = 0; m1 <= p - ms; ++m1) {
      const int len = p - ms - m1 + 1;
      float c = cb[base + len - 1];
      f2_t v = f2pack(c, c), dv = 0ull;
      for (int k = len - 2; k >= 0; --k) {
        if (GRAD) dv = f2fma(dv, U0, v);
        c = cb[base + k];
        v = f2fma(v, U0, f2pack(c, c));
      }
      const f2_t vy = f2mul(v, py);
      far = f2fma(vy, pz, far);
      if (GRAD) {
        gf[0] = f2fma(f2mul(dv, py), pz, gf[0]);
        gf[1] = f2fma(f2mul(v, pym), pz, gf[1]);
        gf[2] = f2fma(vy, pzm, gf[2]);
      }
      pym = f2fma(pym, U1, py);
      py = f2mul(py, U1);
      base += len;
    }
    pzm = f2fma(pzm, U2, pz);
    pz = f2mul(pz, U2);
  }
  return far;
}

// Far field (L2P) added to the near field already in phi/grad.  A warp takes
// two target leaves, one per half; lane l of a half evaluates targets l and
// l + 16 of a 32-target block as the two halves of packed f32x2 operations,
// which halves the instructions a target costs (the evaluation is bound by
// instruction issue, not memory).  Each half-warp first decompresses its leaf's local expansion (FP64) into
// N(p) float coefficients with 1/m! in shared memory -- the coefficients feed
// float arithmetic, so the short, O(1)-coefficient recurrence runs in float
// as well -- then evaluates.
template <bool GRAD>
__global__ void __launch_bounds__(32 * kFastWarps) k_leaf_far(
    PlanDev pd, const Geom* __restrict__ g, int64_t nleaf, const double* __restrict__ lc,
    const int* __restrict__ tstart, const float4* __restrict__ txr, const int* __restrict__ tperm,
    double* __restrict__ phi, double* __restrict__ grad) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, l16 = lane & 15, half = lane >> 4;
  const int64_t b = ((int64_t)blockIdx.x * kFastWarps + warp) * 2 + half;
  if (b - half >= nleaf) return;  // warp-uniform: no leaf for either half
  const bool has = b < nleaf;
  const int64_t bl = has ? b : nleaf - 1;  // a leaf without targets still runs the sweep
  const int t0 = has ? tstart[b] : 0, t1 = has ? tstart[b + 1] : 0;
  extern __shared__ __align__(16) float dsm[];
  const int pitch = (pd.nfull + 1) | 1;  // odd pitch: the halves' rows start in different banks
  float* Dt = dsm + (size_t)(2 * warp + half) * pitch;
  {
    const int nt = pd.nterms > 0 ? pd.nterms : 1;
    float cf[FMM_MAX_TERMS];
    for (int t = 0; t < pd.nterms; ++t) cf[t] = scaled_coef_t<float>(pd, t, g->s_leaf);
    for (int q = l16; q < pd.nj; q += 16) Dt[q] = (float)lc[(size_t)bl * pd.nj + q];
    __syncwarp();
    for (int ms = pd.c; ms <= pd.p; ++ms) {  // the same sweep in both halves
      const int b0 = slab_begin(pd, ms), b1 = slab_begin(pd, ms + 1);
      for (int i = b0 + l16; i < b1; i += 16) {
        float v = 0.f;
        for (int t = 0; t < pd.nterms; ++t) v += cf[t] * Dt[pd.rec_src[i * nt + t]];
        Dt[i] = v;
      }
      __syncwarp();
    }
    for (int q = l16; q < pd.nfull; q += 16) Dt[q] *= pd.inv_fact_f[q];
    __syncwarp();
  }
  const float* cb = Dt;
  const double inv_s = g->inv_s_leaf;
  for (int tb = t0; tb < t1; tb += 32) {
    const int ta = tb + l16, tc = tb + 16 + l16;
    const bool va = ta < t1, vc = tc < t1;
    const float4 qa = va ? txr[ta] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 qc = vc ? txr[tc] : make_float4(0.f, 0.f, 0.f, 0.f);
    f2_t gf[3] = {0ull, 0ull, 0ull};
    const f2_t far = far_field2<GRAD>(pd, cb, f2pack(qa.x, qc.x), f2pack(qa.y, qc.y),
                                      f2pack(qa.z, qc.z), gf);
    float fa, fc;
    f2unpack(far, fa, fc);
    float ga[3], gc[3];
    if (GRAD)
      for (int k = 0; k < 3; ++k) f2unpack(gf[k], ga[k], gc[k]);
    if (va) {
      const int orig = tperm[ta];
      if (phi) phi[orig] += (double)fa;
      if (GRAD && grad)
        for (int k = 0; k < 3; ++k) grad[(size_t)orig * 3 + k] += (double)ga[k] * inv_s;
    }
    if (vc) {
      const int orig = tperm[tc];
      if (phi) phi[orig] += (double)fc;
      if (GRAD && grad)
        for (int k = 0; k < 3; ++k) grad[(size_t)orig * 3 + k] += (double)gc[k] * inv_s;
    }
  }
}

template <int K>
void near_fast_launch(const fmm_plan_s* P, const Workspace& ws, double* phi, double* grad,
                      cudaStream_t st) {
  const PlanDev& pd = P->pd;
  const int L = P->desc.levels;
  const int64_t nleaf = nbox_at(3, L);
  const unsigned nbk = (unsigned)((nleaf + kFastWarps - 1) / kFastWarps);
  if (grad)
    k_leaf_fast<K, true><<<nbk, 32 * kFastWarps, 0, st>>>(
        pd, ws.geom, L, nleaf, ws.tstart, ws.txr, ws.tperm, ws.sstart, ws.sxr, phi, grad);
  else
    k_leaf_fast<K, false><<<nbk, 32 * kFastWarps, 0, st>>>(
        pd, ws.geom, L, nleaf, ws.tstart, ws.txr, ws.tperm, ws.sstart, ws.sxr, phi, grad);
}

template <int K, int D, typename T>
void leaf_launch(const fmm_plan_s* P, const Workspace& ws, double* phi, double* grad,
                 cudaStream_t st) {
  if (grad) leaf_launch_g<K, D, T, true>(P, ws, phi, grad, st);
  else leaf_launch_g<K, D, T, false>(P, ws, phi, grad, st);
}

// ---------------------------------------------------------------------------
// Adaptive tree, FP64: one block per leaf holding targets; each thread owns
// targets and walks the leaf's lists itself (the walk is identical across
// the block):
//   L2P from the leaf's local expansion (levels >= 2);
//   U: coarser adjacent leaves (neighbours of each ancestor at its level),
//      the leaf's colleagues that are leaves, and the finer adjacent leaves
//      found by descending the non-leaf colleagues -> P2P (eq. (1));
//   W: the boxes met in that descent that are not adjacent to the leaf
//      (their parent is) -> M2P, sum_q Ht_q((x - c_C)/s_C) bt_C[q], or P2P
//      when the box holds at most |j| sources;
//   X pairs of the leaf and its ancestors holding at most |j| targets -> P2P
//      (the P2L pass leaves those boxes out).
// ---------------------------------------------------------------------------
constexpr int kAThreads = 64;
constexpr int kAStack = 8 * (FMM_MAX_ADEPTH + 1);

// X pairs summed directly: for the leaf b (level l, coordinates bc) and each
// ancestor C of level >= 2 holding at most nj targets in its subtree, the
// leaves A of X(C) -- coarser than C, adjacent to C's parent, not adjacent to
// C; each is a neighbour of C's ancestor at A's own level -- send their
// sources to b's targets through p2p(A) (the P2L pass skips such C).
template <typename F>
__device__ void x_direct(const ATree& t, int b, int l, const int* bc, int nj, F&& p2p) {
  int lc = l;
  for (int C = b; C >= 0 && lc >= 2 && t.t1[C] - t.t0[C] <= nj; C = t.par[C], --lc) {
    const int cc[3] = {bc[0] >> (l - lc), bc[1] >> (l - lc), bc[2] >> (l - lc)};
    const int pc[3] = {cc[0] >> 1, cc[1] >> 1, cc[2] >> 1};
    for (int lp = lc - 1; lp >= 0; --lp) {
      const int an[3] = {cc[0] >> (lc - lp), cc[1] >> (lc - lp), cc[2] >> (lc - lp)};
      for (int nb = 0; nb < 27; ++nb) {
        const int nc[3] = {an[0] + nb % 3 - 1, an[1] + (nb / 3) % 3 - 1, an[2] + nb / 9 - 1};
        const int A = alookup(t, lp, nc);
        if (A < 0 || !t.leaf[A]) continue;
        if (aadjacent(lp, nc, lc - 1, pc) && !aadjacent(lp, nc, lc, cc)) p2p(A);
      }
    }
  }
}

__device__ __forceinline__ double green3(int kern, double lam, double r2) {
  const double ri = rsqrt(r2);
  if (kern == FMM_KERNEL_LAPLACE) return ri * (1.0 / (4.0 * 3.14159265358979323846));
  if (kern == FMM_KERNEL_YUKAWA) return exp(-lam * r2 * ri) * ri;
  return r2 * ri;  // biharmonic: r
}

__global__ void __launch_bounds__(kAThreads) k_aleaf(
    PlanDev pd, const Geom* __restrict__ g, ATree t, const double* __restrict__ lc,
    const double* __restrict__ mp, const double* __restrict__ tx0, const double* __restrict__ tx1,
    const double* __restrict__ tx2, const int* __restrict__ tperm, const double* __restrict__ sx0,
    const double* __restrict__ sx1, const double* __restrict__ sx2, const double* __restrict__ sw,
    double* __restrict__ phi, int* __restrict__ err) {
  const int b = blockIdx.x;
  if (b >= t.loff[t.maxlev + 1] || !t.leaf[b] || t.t1[b] == t.t0[b]) return;
  const int p = pd.p, nfull = pd.nfull;
  int l, bc[3];
  abox(t, b, &l, bc);
  double cb[3], s;
  abox_center(g, l, bc, cb, &s);
  extern __shared__ __align__(16) double smd[];
  double* a = smd;  // decompressed local / m!
  const int sl = min(pd.c, p + 1) * (p + 1);
  const int per = (kernel_screened(pd.kernel) ? 6 : 3) * sl;
  double* S = smd + ((nfull + 1) & ~1) + threadIdx.x * per;
  const bool has_local = l >= 2;
  if (has_local) {
    for (int q = threadIdx.x; q < pd.nj; q += blockDim.x) a[q] = lc[(size_t)b * pd.nj + q];
    __syncthreads();
    decompress_smem<double>(pd, a, s);
    for (int q = threadIdx.x; q < nfull; q += blockDim.x) a[q] *= pd.inv_fact[q];
    __syncthreads();
  }
  const double inv_s = 1.0 / s, lam = pd.lam;
  const int kern = pd.kernel;
  for (int ti = t.t0[b] + threadIdx.x; ti < t.t1[b]; ti += blockDim.x) {
    const double x[3] = {tx0[ti], tx1[ti], tx2[ti]};
    double acc = 0.0;
    if (has_local) {  // L2P, Sec. 3.3
      double pw[3][FMM_MAXP + 1];
      for (int k = 0; k < 3; ++k) {
        const double u = (x[k] - cb[k]) * inv_s;
        pw[k][0] = 1.0;
        for (int e = 1; e <= p; ++e) pw[k][e] = pw[k][e - 1] * u;
      }
      for (int q = 0; q < nfull; ++q) {
        const char4 m = pd.mi[q];
        acc += a[q] * pw[0][m.x] * pw[1][m.y] * pw[2][m.z];
      }
    }
    auto p2p = [&](int A) {
      for (int q = t.s0[A]; q < t.s1[A]; ++q) {
        const double d0 = x[0] - sx0[q], d1 = x[1] - sx1[q], d2 = x[2] - sx2[q];
        const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
        if (r2 > 0.0) acc += sw[q] * green3(kern, lam, r2);
      }
    };
    auto m2p = [&](int C, int lc_, const int* cc) {
      double c2[3], s2;
      abox_center(g, lc_, cc, c2, &s2);
      const double is2 = 1.0 / s2;
      const double y[3] = {(x[0] - c2[0]) * is2, (x[1] - c2[1]) * is2, (x[2] - c2[2]) * is2};
      const double* bt = mp + (size_t)C * pd.nj;
      double v = 0.0;
      deriv_point(pd, y, lam * s2, deriv_scale(pd, s2), S, sl,
                  [&](int pos, double h) { v += h * bt[pos]; });
      acc += v;
    };
    // U: coarser adjacent leaves
    for (int lp = l - 1; lp >= 0; --lp) {
      const int an[3] = {bc[0] >> (l - lp), bc[1] >> (l - lp), bc[2] >> (l - lp)};
      for (int nb = 0; nb < 27; ++nb) {
        const int nc[3] = {an[0] + nb % 3 - 1, an[1] + (nb / 3) % 3 - 1, an[2] + nb / 9 - 1};
        const int A = alookup(t, lp, nc);
        if (A >= 0 && t.leaf[A] && aadjacent(lp, nc, l, bc)) p2p(A);
      }
    }
    // colleagues: leaves -> U; others -> descend (adjacent: deeper, else W)
    for (int nb = 0; nb < 27; ++nb) {
      const int nc[3] = {bc[0] + nb % 3 - 1, bc[1] + (nb / 3) % 3 - 1, bc[2] + nb / 9 - 1};
      const int C = alookup(t, l, nc);
      if (C < 0) continue;
      if (t.leaf[C]) {
        p2p(C);
        continue;
      }
      int stack[kAStack];
      int sp = 0;
      for (int ci = 0; ci < 8; ++ci)
        if (t.child[8 * C + ci] >= 0) stack[sp++] = t.child[8 * C + ci];
      while (sp > 0) {
        const int E = stack[--sp];
        int le, ce[3];
        abox(t, E, &le, ce);
        if (!aadjacent(le, ce, l, bc)) {
          if (t.s1[E] - t.s0[E] <= pd.nj) p2p(E);  // W box of at most |j| sources
          else m2p(E, le, ce);
        } else if (t.leaf[E]) {
          p2p(E);
        } else {
          for (int ci = 0; ci < 8; ++ci) {
            const int F = t.child[8 * E + ci];
            if (F < 0) continue;
            if (sp < kAStack) stack[sp++] = F;
            else atomicOr(err, 4);  // cannot happen: depth-first, 7 siblings per level
          }
        }
      }
    }
    x_direct(t, b, l, bc, pd.nj, p2p);
    phi[tperm[ti]] = acc;
  }
}

}  // namespace

cudaError_t launch_leaf_eval(const fmm_plan_s* P, const Workspace& ws, double* phi, double* grad,
                             cudaStream_t st, int* nl) {
  const bool f64 = P->desc.precision == FMM_PREC_FP64;
  const int k = P->pd.kernel, d = P->pd.d;
  if (!f64 && d == 3) {  // near field, then far field, on one stream
    cudaError_t e = launch_near_field(P, ws, phi, grad, st, nl);
    if (e != cudaSuccess) return e;
    return launch_far_field(P, ws, phi, grad, st, nl);
  }
  if (d == 2 && k == FMM_KERNEL_BIHARMONIC) {
    if (f64) leaf_launch<FMM_KERNEL_BIHARMONIC, 2, double>(P, ws, phi, grad, st);
    else leaf_launch<FMM_KERNEL_BIHARMONIC, 2, float>(P, ws, phi, grad, st);
  } else if (d == 2) {
    if (f64) leaf_launch<FMM_KERNEL_LAPLACE, 2, double>(P, ws, phi, grad, st);
    else leaf_launch<FMM_KERNEL_LAPLACE, 2, float>(P, ws, phi, grad, st);
  } else if (k == FMM_KERNEL_LAPLACE) {
    leaf_launch<FMM_KERNEL_LAPLACE, 3, double>(P, ws, phi, grad, st);
  } else if (k == FMM_KERNEL_YUKAWA) {
    leaf_launch<FMM_KERNEL_YUKAWA, 3, double>(P, ws, phi, grad, st);
  } else if (k == FMM_KERNEL_HELMHOLTZ) {
    leaf_launch<FMM_KERNEL_HELMHOLTZ, 3, double>(P, ws, phi, grad, st);
  } else if (k == kHelmIm) {
    leaf_launch<kHelmIm, 3, double>(P, ws, phi, grad, st);
  } else {
    leaf_launch<FMM_KERNEL_BIHARMONIC, 3, double>(P, ws, phi, grad, st);
  }
  ++*nl;
  return cudaGetLastError();
}


cudaError_t launch_adaptive_leaf(const fmm_plan_s* P, const Workspace& ws, const ATree& t,
                                 double* phi, cudaStream_t st, int* nl) {
  const PlanDev& pd = P->pd;
  const int nbox = t.loff[t.maxlev + 1];
  if (P->desc.precision != FMM_PREC_FP64) return launch_adaptive_leaf_warp(P, ws, t, phi, st, nl);
  const int sl = std::min(pd.c, pd.p + 1) * (pd.p + 1);
  const int per = (kernel_screened(pd.kernel) ? 6 : 3) * sl;
  const size_t smem = sizeof(double) * (((pd.nfull + 1) & ~1) + (size_t)per * kAThreads);
  set_smem(k_aleaf, smem);
  k_aleaf<<<(unsigned)nbox, kAThreads, smem, st>>>(pd, ws.geom, t, ws.lc, ws.mp, ws.tx[0],
                                                   ws.tx[1], ws.tx[2], ws.tperm, ws.sx[0],
                                                   ws.sx[1], ws.sx[2], ws.sw, phi,
                                                   &ws.geom->flag);
  ++*nl;
  return cudaGetLastError();
}

// Split leaf pass of the FP32 3D path: the near field alone (to be launched
// on a second stream as soon as the points are sorted) ...
bool leaf_split_supported(const fmm_plan_s* P) {
  return P->desc.precision != FMM_PREC_FP64 && P->pd.d == 3 && P->desc.levels > 0;
}

cudaError_t launch_near_field(const fmm_plan_s* P, const Workspace& ws, double* phi,
                              double* grad, cudaStream_t st, int* nl) {
  const int k = P->pd.kernel;
  if (k == FMM_KERNEL_LAPLACE) near_fast_launch<FMM_KERNEL_LAPLACE>(P, ws, phi, grad, st);
  else if (k == FMM_KERNEL_YUKAWA) near_fast_launch<FMM_KERNEL_YUKAWA>(P, ws, phi, grad, st);
  else if (k == FMM_KERNEL_HELMHOLTZ) near_fast_launch<FMM_KERNEL_HELMHOLTZ>(P, ws, phi, grad, st);
  else if (k == kHelmIm) near_fast_launch<kHelmIm>(P, ws, phi, grad, st);
  else near_fast_launch<FMM_KERNEL_BIHARMONIC>(P, ws, phi, grad, st);
  ++*nl;
  return cudaGetLastError();
}

// ... and the far field added afterwards (leaf coefficients, then L2P)
cudaError_t launch_far_field(const fmm_plan_s* P, const Workspace& ws, double* phi,
                             double* grad, cudaStream_t st, int* nl) {
  const PlanDev& pd = P->pd;
  if (launch_l2p_f32(P, ws, phi, grad, st)) {  // orders with the warp-per-leaf kernel
    ++*nl;
    return cudaGetLastError();
  }
  const int L = P->desc.levels;
  const int64_t nleaf = nbox_at(3, L);
  const double* lcL = ws.lc + ws.lev_off[L] * pd.nj;
  const size_t sm = sizeof(float) * (size_t)((pd.nfull + 1) | 1) * 2 * kFastWarps;
  const unsigned nbk = (unsigned)((nleaf + 2 * kFastWarps - 1) / (2 * kFastWarps));
  if (grad) {
    set_smem(k_leaf_far<true>, sm);
    k_leaf_far<true><<<nbk, 32 * kFastWarps, sm, st>>>(pd, ws.geom, nleaf, lcL, ws.tstart,
                                                       ws.txr, ws.tperm, phi, grad);
  } else {
    set_smem(k_leaf_far<false>, sm);
    k_leaf_far<false><<<nbk, 32 * kFastWarps, sm, st>>>(pd, ws.geom, nleaf, lcL, ws.tstart,
                                                        ws.txr, ws.tperm, phi, grad);
  }
  ++*nl;
  return cudaGetLastError();
}
