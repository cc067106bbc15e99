// Device helpers shared by the expansion kernels: box geometry, slab ranges,
// and the sparse decompression / compression sweeps of Thm 4.
#pragma once

#include "dwf.cuh"
#include "fmm_internal.cuh"

// number of rows of the full layout and the start of slab ms
__device__ __forceinline__ int slab_begin(const PlanDev& pd, int ms) {
  if (ms > pd.p) return pd.nfull;
  return pd.d == 3 ? pd.frow[ms * (pd.p + 1)] : pd.frow[ms];
}

// 2^-e for 0 <= e <= 126, exact, from the exponent field (no FP64 work in
// float kernels)
template <typename T>
__device__ __forceinline__ T pow2_neg(int e);
template <>
__device__ __forceinline__ float pow2_neg<float>(int e) {
  return __int_as_float((127 - e) << 23);
}
template <>
__device__ __forceinline__ double pow2_neg<double>(int e) {
  return __longlong_as_double((long long)(1023 - e) << 52);
}
template <>
__device__ __forceinline__ dwf pow2_neg<dwf>(int e) {
  return dwf(pow2_neg<float>(e), 0.f);
}

// Box centre at level l (lexicographic index b, x fastest), round-to-nearest
// operations in the same order as lo + (b + 1/2) * s.
template <int D>
__device__ __forceinline__ void box_center(const Geom* g, int l, int64_t b, int* bc, double* c,
                                           double* s_out) {
  const int nl = 1 << l;
  const double s = __dmul_rn(g->size, pow2_neg<double>(l));  // size / 2^l, exact
  for (int k = 0; k < D; ++k) {
    bc[k] = (int)(b % nl);
    b /= nl;
    c[k] = __dadd_rn(g->lo[k], __dmul_rn((double)bc[k] + 0.5, s));
  }
  *s_out = s;
}

// scaled recurrence coefficients at box side s: a_xi s^{c-|xi|} (eq. (define_pde_op)
// in units of the box side)
__device__ __forceinline__ double scaled_coef(const PlanDev& pd, int t, double s) {
  double v = pd.tcoef[t];
  for (int k = 0; k < pd.tpow[t]; ++k) v *= s;
  return v;
}

// the scaled coefficient in the kernel's arithmetic: float kernels take the
// float copy when no power of s enters (every term of the PDE's order c, as
// for the Laplace and biharmonic operators), so that no FP64 work is done
template <typename T>
__device__ __forceinline__ T scaled_coef_t(const PlanDev& pd, int t, double s);
template <>
__device__ __forceinline__ double scaled_coef_t<double>(const PlanDev& pd, int t, double s) {
  return scaled_coef(pd, t, s);
}
template <>
__device__ __forceinline__ float scaled_coef_t<float>(const PlanDev& pd, int t, double s) {
  return pd.tpow[t] == 0 ? pd.tcoef_f[t] : (float)scaled_coef(pd, t, s);
}
template <>
__device__ __forceinline__ dwf scaled_coef_t<dwf>(const PlanDev& pd, int t, double s) {
  return dwf(scaled_coef(pd, t, s));
}
// 1/m! in the kernel's arithmetic
template <typename T>
__device__ __forceinline__ T inv_fact_t(const PlanDev& pd, int q);
template <>
__device__ __forceinline__ double inv_fact_t<double>(const PlanDev& pd, int q) {
  return pd.inv_fact[q];
}
template <>
__device__ __forceinline__ float inv_fact_t<float>(const PlanDev& pd, int q) {
  return pd.inv_fact_f[q];
}
template <>
__device__ __forceinline__ dwf inv_fact_t<dwf>(const PlanDev& pd, int q) {
  return dwf(pd.inv_fact[q]);
}

// warp shuffle of a float, double or double-word value
__device__ __forceinline__ float shfl_t(float v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}
__device__ __forceinline__ double shfl_t(double v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}
__device__ __forceinline__ dwf shfl_t(dwf v, int src) {
  return dwf(__shfl_sync(0xffffffffu, v.h, src), __shfl_sync(0xffffffffu, v.l, src));
}

// The scaled recurrence coefficients of a block's sweep: computed once, by
// the first nterms threads (FP64 work, 1/64 of the FP32 rate on this GPU),
// into shared memory; the caller synchronises before reading.
template <typename T>
__device__ __forceinline__ const T* block_coefs(const PlanDev& pd, double s) {
  __shared__ T cs[FMM_MAX_TERMS];
  if (threadIdx.x < pd.nterms) cs[threadIdx.x] = scaled_coef_t<T>(pd, threadIdx.x, s);
  return cs;
}
// the same for a warp: lane t computes coefficient t, shuffled to all lanes
template <typename T>
__device__ __forceinline__ void warp_coefs(const PlanDev& pd, double s, int lane, T* coef) {
  const T mine = lane < pd.nterms ? scaled_coef_t<T>(pd, lane, s) : T(0);
  for (int t = 0; t < pd.nterms; ++t) coef[t] = shfl_t(mine, t);
}

// D[j] given in a[0..nj); fill slabs c..p (decompression, eq. (decompression)).
template <typename T>
__device__ void decompress_smem(const PlanDev& pd, T* a, double s) {
  const int nt = pd.nterms > 0 ? pd.nterms : 1;
  const T* coef = block_coefs<T>(pd, s);
  __syncthreads();
  for (int ms = pd.c; ms <= pd.p; ++ms) {
    const int b0 = slab_begin(pd, ms), b1 = slab_begin(pd, ms + 1);
    for (int i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
      T v = 0;
      for (int t = 0; t < pd.nterms; ++t) v += coef[t] * a[pd.rec_src[i * nt + t]];
      a[i] = v;
    }
    __syncthreads();
  }
}

// alpha in a[0..nfull); on return a[0..nj) = M^T alpha (eq. (define_beta_multipole)),
// swept from the top slab down in gather form.
template <typename T>
__device__ void compress_smem(const PlanDev& pd, T* a, double s) {
  const int nt = pd.nterms > 0 ? pd.nterms : 1;
  const T* coef = block_coefs<T>(pd, s);
  __syncthreads();
  for (int ms = pd.p - 1; ms >= 0; --ms) {
    const int b0 = slab_begin(pd, ms), b1 = slab_begin(pd, ms + 1);
    for (int i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
      T v = a[i];
      for (int t = 0; t < pd.nterms; ++t) {
        const int src = pd.cmp_src[i * nt + t];
        if (src >= 0) v += coef[t] * a[src];
      }
      a[i] = v;
    }
    __syncthreads();
  }
}

template <typename T>
__host__ __device__ __forceinline__ size_t align_bytes(size_t n) {
  return (n + 15) / 16 * 16;
}

// Warp-synchronous version of compress_smem: one warp owns `a`.
template <typename T>
__device__ void compress_warp(const PlanDev& pd, T* a, double s, int lane) {
  const int nt = pd.nterms > 0 ? pd.nterms : 1;
  T coef[FMM_MAX_TERMS];
  warp_coefs<T>(pd, s, lane, coef);
  for (int ms = pd.p - 1; ms >= 0; --ms) {
    const int b0 = slab_begin(pd, ms), b1 = slab_begin(pd, ms + 1);
    for (int i = b0 + lane; i < b1; i += 32) {
      T v = a[i];
      for (int t = 0; t < pd.nterms; ++t) {
        const int src = pd.cmp_src[i * nt + t];
        if (src >= 0) v += coef[t] * a[src];
      }
      a[i] = v;
    }
    __syncwarp();
  }
}

// Warp-synchronous version of decompress_smem: one warp owns `a`.
template <typename T>
__device__ void decompress_warp(const PlanDev& pd, T* a, double s, int lane) {
  const int nt = pd.nterms > 0 ? pd.nterms : 1;
  T coef[FMM_MAX_TERMS];
  warp_coefs<T>(pd, s, lane, coef);
  for (int ms = pd.c; ms <= pd.p; ++ms) {
    const int b0 = slab_begin(pd, ms), b1 = slab_begin(pd, ms + 1);
    for (int i = b0 + lane; i < b1; i += 32) {
      T v = 0;
      for (int t = 0; t < pd.nterms; ++t) v += coef[t] * a[pd.rec_src[i * nt + t]];
      a[i] = v;
    }
    __syncwarp();
  }
}

// Box-scaled derivatives s^{|m|} d^m G at the point s*x (x in box units) for
// the stored set j (order p, slabs m_s < c), degree by degree, from the same
// r^2-led recurrences as the M2L derivative tables (Sec. 4.4; 3D Laplace,
// Yukawa, Helmholtz parts, biharmonic).  Only the last two degrees are kept:
// S holds 3 * sl values (6 * sl for the coupled recurrences),
// sl = min(c, p+1) * (p+1), private to the
// caller.  emit(pos, value) receives value * scale for the multi-index at
// position pos of the stored layout.  lam is lambda * s.  T = double, or
// float for the mixed-precision modes.
template <typename T, typename F>
__device__ void deriv_point(const PlanDev& pd, const T* x, T lam, T scale, T* S, int sl,
                            F&& emit) {
  const int p = pd.p, ce = pd.c < p + 1 ? pd.c : p + 1;
  const bool yuk = kernel_screened(pd.kernel);
  const T nu = pd.kernel == FMM_KERNEL_BIHARMONIC ? T(1) : T(-1);
  const T alpha = pd.kernel == kHelmIm ? lam : -lam;  // coupled recurrence (see the tables)
  const T beta = pd.kernel == FMM_KERNEL_HELMHOLTZ ? lam : -lam;
  const T r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  const T r = sqrt(r2), rinv2 = T(1) / r2;
  T* G3[3] = {S, S + sl, S + 2 * sl};
  T* B3[3] = {S + 3 * sl, S + 4 * sl, S + 5 * sl};
  if (pd.kernel == FMM_KERNEL_YUKAWA) {
    const T e = exp(-lam * r);
    G3[0][0] = e / r;
    B3[0][0] = e;
  } else if (yuk) {
    const T sn = sin(lam * r), cs = cos(lam * r);
    G3[0][0] = (pd.kernel == FMM_KERNEL_HELMHOLTZ ? cs : sn) / r;
    B3[0][0] = pd.kernel == FMM_KERNEL_HELMHOLTZ ? sn : cs;
  } else {
    G3[0][0] = pd.kernel == FMM_KERNEL_BIHARMONIC ? r : T(1) / r;
  }
  emit(0, G3[0][0] * scale);
  for (int n = 1; n <= p; ++n) {
    T* cur = G3[n % 3];
    const T* g1s = G3[(n + 2) % 3];  // degree n-1
    const T* g2s = G3[(n + 1) % 3];  // degree n-2
    T* bcur = B3[n % 3];
    const T* b1s = B3[(n + 2) % 3];
    const T* b2s = B3[(n + 1) % 3];
    for (int ms = 0; ms < ce && ms <= n; ++ms) {
      for (int m1 = 0; m1 <= n - ms; ++m1) {
        const int m[3] = {n - ms - m1, m1, ms};
        int a = 0;
        while (m[a] == 0) ++a;
        const int ma = m[a];
        // position of a multi-index q of degree dq in its slice
        auto pos = [](int dq, int qs, int q1) { return qs * (dq + 1) - qs * (qs - 1) / 2 + q1; };
        int q1[3] = {m[0], m[1], m[2]};
        q1[a] -= 1;
        const T g1 = g1s[pos(n - 1, q1[2], q1[1])];
        T g2 = 0, b1 = 0, b2 = 0;
        if (yuk) b1 = b1s[pos(n - 1, q1[2], q1[1])];
        if (ma >= 2) {
          int q2[3] = {m[0], m[1], m[2]};
          q2[a] -= 2;
          g2 = g2s[pos(n - 2, q2[2], q2[1])];
          if (yuk) b2 = b2s[pos(n - 2, q2[2], q2[1])];
        }
        T v;
        if (yuk)
          v = -(T(2) * ma - T(1)) * x[a] * g1 - T((ma - 1) * (ma - 1)) * g2 +
              alpha * x[a] * b1 + alpha * T(ma - 1) * b2;
        else
          v = (nu - T(2 * (ma - 1))) * x[a] * g1 + T(ma - 1) * (nu - T(ma - 2)) * g2;
        for (int bax = a + 1; bax < 3; ++bax) {
          const int mb = m[bax];
          if (mb == 0) continue;
          int qb[3] = {m[0], m[1], m[2]};
          qb[bax] -= 1;
          v -= T(2 * mb) * x[bax] * g1s[pos(n - 1, qb[2], qb[1])];
          if (mb >= 2) {
            qb[bax] -= 1;
            v -= T(mb * (mb - 1)) * g2s[pos(n - 2, qb[2], qb[1])];
          }
        }
        const int pm = pos(n, ms, m1);
        cur[pm] = v * rinv2;
        if (yuk) bcur[pm] = beta * (x[a] * g1 + T(ma - 1) * g2);
        emit(pd.frow[ms * (p + 1) + m1] + m[0], cur[pm] * scale);
      }
    }
  }
}

// scale of the box-scaled derivatives at side s (3D kernels)
__device__ inline double deriv_scale(const PlanDev& pd, double s) {
  if (pd.kernel == FMM_KERNEL_LAPLACE) return 1.0 / (4.0 * 3.14159265358979323846 * s);
  if (pd.kernel == FMM_KERNEL_BIHARMONIC) return s;
  return 1.0 / s;  // Yukawa, Helmholtz parts
}
