// Device helpers shared by the expansion kernels: box geometry, slab ranges,
// and the sparse decompression / compression sweeps of Thm 4.
#pragma once

#include "fmm_internal.cuh"

// number of rows of the full layout and the start of slab ms
__device__ __forceinline__ int slab_begin(const PlanDev& pd, int ms) {
  if (ms > pd.p) return pd.nfull;
  return pd.d == 3 ? pd.frow[ms * (pd.p + 1)] : pd.frow[ms];
}

// Box centre at level l (lexicographic index b, x fastest), round-to-nearest
// operations in the same order as lo + (b + 1/2) * s.
template <int D>
__device__ __forceinline__ void box_center(const Geom* g, int l, int64_t b, int* bc, double* c,
                                           double* s_out) {
  const int nl = 1 << l;
  const double s = __ddiv_rn(g->size, (double)nl);
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

// D[j] given in a[0..nj); fill slabs c..p (decompression, eq. (decompression)).
template <typename T>
__device__ void decompress_smem(const PlanDev& pd, T* a, double s) {
  const int nt = pd.nterms > 0 ? pd.nterms : 1;
  T coef[FMM_MAX_TERMS];
  for (int t = 0; t < pd.nterms; ++t) coef[t] = (T)scaled_coef(pd, t, s);
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
  T coef[FMM_MAX_TERMS];
  for (int t = 0; t < pd.nterms; ++t) coef[t] = (T)scaled_coef(pd, t, s);
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
  for (int t = 0; t < pd.nterms; ++t) coef[t] = (T)scaled_coef(pd, t, s);
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
