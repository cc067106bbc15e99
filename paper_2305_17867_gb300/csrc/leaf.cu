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

#include "expansions.cuh"

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
  } else if (K == FMM_KERNEL_YUKAWA) {
    const T ri = rsqrt_t(r2);
    const T r = r2 * ri;
    const T e = exp_t(-lam * r);
    v = e * ri;
    f1 = e * (-lam * ri * ri - ri * ri * ri);
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
    T nv = 0, ng[3] = {0, 0, 0}, wsum = 0;
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
              wsum += wj;
              if (GRAD) {
                const T fw = wj * f1;
                for (int k = 0; k < D; ++k) ng[k] += fw * dxv[k];
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
      } else if (K == FMM_KERNEL_YUKAWA) {
        phi_scale = inv_s;
        grad_scale = inv_s * inv_s;
      } else {
        phi_scale = s;
        grad_scale = 1.0;
      }
      const int orig = tperm[t];
      double ph = (double)far + phi_scale * (double)nv;
      if (K == FMM_KERNEL_LAPLACE && D == 2) ph += log(s) * (double)wsum;
      if (phi) phi[orig] = ph;
      if (GRAD && grad)
        for (int k = 0; k < D; ++k)
          grad[(size_t)orig * D + k] = (double)gf[k] * inv_s + grad_scale * (double)ng[k];
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

template <int K, int D, typename T>
void leaf_launch(const fmm_plan_s* P, const Workspace& ws, double* phi, double* grad,
                 cudaStream_t st) {
  if (grad) leaf_launch_g<K, D, T, true>(P, ws, phi, grad, st);
  else leaf_launch_g<K, D, T, false>(P, ws, phi, grad, st);
}

}  // namespace

cudaError_t launch_leaf_eval(const fmm_plan_s* P, const Workspace& ws, double* phi, double* grad,
                             cudaStream_t st, int* nl) {
  const bool f64 = P->desc.precision == FMM_PREC_FP64;
  const int k = P->pd.kernel, d = P->pd.d;
  if (d == 2) {
    if (f64) leaf_launch<FMM_KERNEL_LAPLACE, 2, double>(P, ws, phi, grad, st);
    else leaf_launch<FMM_KERNEL_LAPLACE, 2, float>(P, ws, phi, grad, st);
  } else if (k == FMM_KERNEL_LAPLACE) {
    if (f64) leaf_launch<FMM_KERNEL_LAPLACE, 3, double>(P, ws, phi, grad, st);
    else leaf_launch<FMM_KERNEL_LAPLACE, 3, float>(P, ws, phi, grad, st);
  } else if (k == FMM_KERNEL_YUKAWA) {
    if (f64) leaf_launch<FMM_KERNEL_YUKAWA, 3, double>(P, ws, phi, grad, st);
    else leaf_launch<FMM_KERNEL_YUKAWA, 3, float>(P, ws, phi, grad, st);
  } else {
    if (f64) leaf_launch<FMM_KERNEL_BIHARMONIC, 3, double>(P, ws, phi, grad, st);
    else leaf_launch<FMM_KERNEL_BIHARMONIC, 3, float>(P, ws, phi, grad, st);
  }
  ++*nl;
  return cudaGetLastError();
}
