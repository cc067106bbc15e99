// Derivative tables (Sec. 4.4), P2M (Sec. 3.4), M2M (Sec. 4.3), L2L (Sec. 4.2).
#include <algorithm>
#include <cmath>
#include <vector>

#include "adaptive.cuh"
#include "expansions.cuh"
#include "passes_f32.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxT = 8;  // full-layout terms per thread: 8 * 256 >= N(20) in 3D

template <typename K>
void set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// ---------------------------------------------------------------------------
// M2L derivative tables.  For every level l >= 2 and every offset h in
// [-3,3]^d outside [-1,1]^d (box units) the block fills
//   Ht[m] = s_l^{|m|} d^m G(s_l h),  m in the Hankel layout (|m| <= 2p, m_s <= 2c-2),
// from r^2-led recurrences obtained, as in Sec. 4.4, by applying the Leibniz
// rule to an identity r^2 d_a g = (...):
//   g = r^nu (3D Laplace nu=-1, 3D biharmonic nu=+1):  r^2 d_a g = nu x_a g
//   g = log r (2D Laplace, eq. (deriv_laplace_2d)):      r^2 d_a g = x_a
//   g = r^2 log r (2D biharmonic):                       r^2 d_a g = 2 x_a g + x_a r^2
//   g = e^{-lam r}/r with b = e^{-lam r} (Yukawa):       r^2 d_a g = -x_a g - lam x_a b,
//                                                         d_a b = -lam x_a g
//   Helmholtz, real part g = cos(k r)/r, b = sin(k r):    r^2 d_a g = -x_a g - k x_a b,
//                                                         d_a b = +k x_a g
//   imaginary part g = sin(k r)/r, b = cos(k r):          r^2 d_a g = -x_a g + k x_a b,
//                                                         d_a b = -k x_a g
// (one coupled form r^2 d_a g = -x_a g + alpha x_a b, d_a b = beta x_a g)
// With a the first axis where m_a >= 1 and k = m - e_a, Leibniz on r^2 gives
//   r^2 g^m = RHS^{(k)} - 2(m_a-1) x_a g^{m-e_a} - (m_a-1)(m_a-2) g^{m-2e_a}
//             - sum_{b != a} [2 m_b x_b g^{m-e_b} + m_b (m_b-1) g^{m-2e_b}],
// which for nu = -1 is the paper's eq. (deriv_laplace_3d).  Every term has
// lower total degree, so the table fills degree by degree.
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ int hidx(const int* hrow, int P2, const int* m) {
  return D == 3 ? hrow[m[2] * (P2 + 1) + m[1]] + m[0] : hrow[m[1]] + m[0];
}

template <int D>
__global__ void __launch_bounds__(128) k_deriv_tables(PlanDev pd, const Geom* __restrict__ g,
                                                      double* __restrict__ htab) {
  constexpr int NOFF = D == 3 ? 343 : 49;
  const int lrel = blockIdx.x / NOFF, o = blockIdx.x % NOFF;
  const int l = lrel + 2;
  double x[3] = {0.0, 0.0, 0.0};
  bool far = false;
  {
    int t = o;
    for (int k = 0; k < D; ++k) {
      const int hk = t % 7 - 3;
      t /= 7;
      x[k] = (double)hk;
      if (hk > 1 || hk < -1) far = true;
    }
  }
  if (!far) return;
  extern __shared__ double sm[];
  double* G = sm;
  double* B = sm + pd.nh;
  __shared__ double sh_r, sh_rinv2;  // one square root and division per block
  const int P2 = 2 * pd.p, nslab = 2 * pd.c - 1;
  const double s = __dmul_rn(g->size, pow2_neg<double>(l));
  if (threadIdx.x == 0) {
    const double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    sh_r = sqrt(r2);
    sh_rinv2 = 1.0 / r2;
  }
  __syncthreads();
  const double r = sh_r, rinv2 = sh_rinv2;
  const int kern = pd.kernel;
  const double lam = pd.lam * s;
  // nu for the r^nu family; log / Yukawa flagged separately
  const bool is_log = (kern == FMM_KERNEL_LAPLACE && D == 2);
  const bool is_bih2 = (kern == FMM_KERNEL_BIHARMONIC && D == 2);
  const bool is_yuk = kernel_screened(kern);
  const double nu = is_bih2 ? 2.0 : (kern == FMM_KERNEL_BIHARMONIC) ? 1.0 : -1.0;
  // coefficients of the coupled recurrence (lam is lambda or kappa, in box units)
  const double alpha = kern == kHelmIm ? lam : -lam;
  const double beta = kern == FMM_KERNEL_HELMHOLTZ ? lam : -lam;
  if (threadIdx.x == 0) {
    if (is_log) {
      G[0] = log(r);
    } else if (is_bih2) {
      G[0] = r * r * log(r);
    } else if (kern == FMM_KERNEL_YUKAWA) {
      const double e = exp(-lam * r);
      G[0] = e / r;
      B[0] = e;
    } else if (is_yuk) {
      double sn, cs;
      sincos(lam * r, &sn, &cs);
      G[0] = (kern == FMM_KERNEL_HELMHOLTZ ? cs : sn) / r;
      B[0] = kern == FMM_KERNEL_HELMHOLTZ ? sn : cs;
    } else {
      G[0] = (kern == FMM_KERNEL_BIHARMONIC) ? r : 1.0 / r;
    }
  }
  __syncthreads();
  for (int deg = 1; deg <= P2; ++deg) {
    int count = 0;
    for (int ms = 0; ms < nslab && ms <= deg; ++ms) count += (D == 3) ? (deg - ms + 1) : 1;
    for (int e = threadIdx.x; e < count; e += blockDim.x) {
      int m[3] = {0, 0, 0};
      {
        int rem = e;
        for (int ms = 0; ms < nslab && ms <= deg; ++ms) {
          const int cnt = (D == 3) ? (deg - ms + 1) : 1;
          if (rem < cnt) {
            if (D == 3) {
              m[2] = ms;
              m[1] = rem;
              m[0] = deg - ms - rem;
            } else {
              m[1] = ms;
              m[0] = deg - ms;
            }
            break;
          }
          rem -= cnt;
        }
      }
      int a = 0;
      while (m[a] == 0) ++a;
      const int ma = m[a];
      int q[3] = {m[0], m[1], m[2]};
      q[a] = ma - 1;
      const int i1 = hidx<D>(pd.hrow, P2, q);
      const double g1 = G[i1];
      double g2 = 0.0, b1 = 0.0, b2 = 0.0;
      int i2 = -1;
      if (ma >= 2) {
        q[a] = ma - 2;
        i2 = hidx<D>(pd.hrow, P2, q);
        g2 = G[i2];
      }
      if (is_yuk) {
        b1 = B[i1];
        if (i2 >= 0) b2 = B[i2];
      }
      double v;
      if (is_log) {
        v = -2.0 * (ma - 1) * x[a] * g1 - (double)(ma - 1) * (ma - 2) * g2;
        if (deg == 1) v += x[a];
        if (deg == 2 && ma == 2) v += 1.0;
      } else if (is_yuk) {
        v = -(2.0 * ma - 1.0) * x[a] * g1 - (double)(ma - 1) * (ma - 1) * g2 +
            alpha * x[a] * b1 + alpha * (ma - 1) * b2;
      } else {
        v = (nu - 2.0 * (ma - 1)) * x[a] * g1 + (double)(ma - 1) * (nu - (ma - 2)) * g2;
        if (is_bih2 && deg <= 4) {
          // + d^k (x_a r^2), k = m - e_a: the monomials x_a^3 and x_a x_b^2
          const int b = 1 - a, ka = ma - 1, kb = m[b];
          auto mono = [&](int ia, int ib) {  // d_a^ka d_b^kb x_a^ia x_b^ib at x
            if (ka > ia || kb > ib) return 0.0;
            double f = 1.0;
            for (int t = 0; t < ka; ++t) f *= ia - t;
            for (int t = 0; t < kb; ++t) f *= ib - t;
            for (int t = 0; t < ia - ka; ++t) f *= x[a];
            for (int t = 0; t < ib - kb; ++t) f *= x[b];
            return f;
          };
          v += mono(3, 0) + mono(1, 2);
        }
      }
      for (int bax = a + 1; bax < D; ++bax) {
        const int mb = m[bax];
        if (mb == 0) continue;
        int qb[3] = {m[0], m[1], m[2]};
        qb[bax] = mb - 1;
        v -= 2.0 * mb * x[bax] * G[hidx<D>(pd.hrow, P2, qb)];
        if (mb >= 2) {
          qb[bax] = mb - 2;
          v -= (double)mb * (mb - 1) * G[hidx<D>(pd.hrow, P2, qb)];
        }
      }
      const int im = hidx<D>(pd.hrow, P2, m);
      G[im] = v * rinv2;
      if (is_yuk) B[im] = beta * (x[a] * g1 + (ma - 1) * g2);
    }
    __syncthreads();
  }
  double scale = 1.0;
  if (kern == FMM_KERNEL_LAPLACE && D == 3) scale = 1.0 / (4.0 * 3.14159265358979323846 * s);
  if (kern == FMM_KERNEL_BIHARMONIC) scale = D == 3 ? s : s * s;
  if (is_yuk) scale = 1.0 / s;
  double* out = htab + ((size_t)lrel * NOFF + o) * pd.nh;
  for (int i = threadIdx.x; i < pd.nh; i += blockDim.x) {
    double v = G[i] * scale;
    if (is_log && i == 0) v += log(s);
    out[i] = v;
  }
  if (is_bih2) {
    // (s r)^2 log(s r) = s^2 (r^2 log r + log(s) r^2): the second part's
    // derivatives, d^m r^2 for |m| <= 2, in units of the box side
    __syncthreads();
    if (threadIdx.x == 0) {
      const double ls = s * s * log(s);
      out[pd.hrow[0]] += ls * (x[0] * x[0] + x[1] * x[1]);
      out[pd.hrow[0] + 1] += ls * 2.0 * x[0];
      out[pd.hrow[0] + 2] += ls * 2.0;
      out[pd.hrow[1]] += ls * 2.0 * x[1];
      out[pd.hrow[2]] += ls * 2.0;
    }
  }
}

// ---------------------------------------------------------------------------
// P2M (Sec. 3.4): per leaf box, alpha_q = sum_y w ((c - y)/s)^q / q!, then
// beta = M^T alpha (compressed, box-scaled).  One block per leaf box.
// ---------------------------------------------------------------------------
template <int D, typename T>
__global__ void __launch_bounds__(kThreads) k_p2m(PlanDev pd, const Geom* __restrict__ g, int L,
                                                  const int* __restrict__ start,
                                                  const double* __restrict__ x0,
                                                  const double* __restrict__ x1,
                                                  const double* __restrict__ x2,
                                                  const double* __restrict__ w,
                                                  const float4* __restrict__ rel,
                                                  double* __restrict__ mp) {
  constexpr int CH = 32;
  const int b = blockIdx.x;
  const int i0 = start[b], i1 = start[b + 1];
  const int p = pd.p, nfull = pd.nfull, nj = pd.nj;
  if (i0 == i1) {
    for (int q = threadIdx.x; q < nj; q += blockDim.x) mp[(size_t)b * nj + q] = 0.0;
    return;
  }
  extern __shared__ __align__(16) unsigned char smraw[];
  T* pw = reinterpret_cast<T*>(smraw);
  T* alpha = reinterpret_cast<T*>(smraw + align_bytes<T>(sizeof(T) * CH * D * (p + 1)));
  int bc[3];
  double c[3] = {0.0, 0.0, 0.0}, s = g->s_leaf;
  if (!rel) box_center<D>(g, L, b, bc, c, &s);
  const double inv_s = rel ? 0.0 : 1.0 / s;  // only the FP64-input path divides
  T acc[kMaxT];
  char4 mt[kMaxT];
#pragma unroll
  for (int k = 0; k < kMaxT; ++k) {
    const int q = threadIdx.x + k * blockDim.x;
    acc[k] = 0;
    mt[k] = q < nfull ? pd.mi[q] : make_char4(0, 0, 0, 0);
  }
  const double* xs[3] = {x0, x1, x2};
  for (int base = i0; base < i1; base += CH) {
    const int n = min(CH, i1 - base);
    __syncthreads();
    if (threadIdx.x < CH * D) {
      const int j = threadIdx.x / D, k = threadIdx.x % D;
      T* row = pw + (j * D + k) * (p + 1);
      if (j < n) {
        T u, v;
        if (rel) {  // (c - y)/s = -(y - c)/s from the box-relative copy
          const float4 r = rel[base + j];
          u = (T)(-(k == 0 ? r.x : (k == 1 ? r.y : r.z)));
          v = (k == 0) ? (T)r.w : (T)1;
        } else {
          u = (T)((c[k] - xs[k][base + j]) * inv_s);
          v = (k == 0) ? (T)w[base + j] : (T)1;
        }
        row[0] = v;
        for (int e = 1; e <= p; ++e) {
          v *= u;
          row[e] = v;
        }
      } else {
        for (int e = 0; e <= p; ++e) row[e] = 0;
      }
    }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
      const T* r0 = pw + j * D * (p + 1);
#pragma unroll
      for (int k = 0; k < kMaxT; ++k) {
        if (threadIdx.x + k * blockDim.x < nfull) {
          T v = r0[mt[k].x] * r0[(p + 1) + mt[k].y];
          if (D == 3) v *= r0[2 * (p + 1) + mt[k].z];
          acc[k] += v;
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kMaxT; ++k) {
    const int q = threadIdx.x + k * blockDim.x;
    if (q < nfull) alpha[q] = acc[k] * inv_fact_t<T>(pd, q);
  }
  __syncthreads();
  compress_smem<T>(pd, alpha, s);
  for (int q = threadIdx.x; q < nj; q += blockDim.x) mp[(size_t)b * nj + q] = (double)alpha[q];
}

// P2M, one warp per leaf box (used when N(p) <= 32 * kWarpTerms).  Lane j of
// a 32-source chunk builds the power table of its source (weight folded into
// the first axis); lane t then accumulates terms q = t, t+32, ...; the
// compression sweep runs warp-synchronously.
constexpr int kWarpTerms = 32;
constexpr int kP2mWarps = 4;

// body of the warp P2M for a box of centre c and side s with sources i0..i1
// of the sorted arrays; writes the compressed box-scaled multipole to out
template <int D, typename T, int NT>
__device__ void p2m_warp_body(const PlanDev& pd, const double* c, double s, int i0, int i1,
                              const double* __restrict__ x0, const double* __restrict__ x1,
                              const double* __restrict__ x2, const double* __restrict__ w,
                              const float4* __restrict__ rel, T* pw, T* alpha, int lane,
                              double* __restrict__ out) {
  const int p = pd.p, nfull = pd.nfull, nj = pd.nj;
  const int P1 = p + 1;
  const double inv_s = rel ? 0.0 : 1.0 / s;  // only the FP64-input path divides
  const int nt = (nfull + 31) / 32;
  T acc[NT];
  int qoff[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    acc[t] = 0;
    const int q = lane + 32 * t;
    qoff[t] = 0;
    if (t < nt && q < nfull) {
      const char4 m = pd.mi[q];
      qoff[t] = m.x | (m.y << 8) | (m.z << 16);
    }
  }
  const double* xs[3] = {x0, x1, x2};
  for (int base = i0; base < i1; base += 32) {
    const int n = min(32, i1 - base);
    __syncwarp();
    {
      T* row = pw + lane * D * P1;
      if (lane < n) {
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
        if (rel) r = rel[base + lane];
        for (int k = 0; k < D; ++k) {
          T u, v;
          if (rel) {  // (c - y)/s = -(y - c)/s from the box-relative copy
            u = (T)(-(k == 0 ? r.x : (k == 1 ? r.y : r.z)));
            v = (k == 0) ? (T)r.w : (T)1;
          } else {
            u = (T)((c[k] - xs[k][base + lane]) * inv_s);
            v = (k == 0) ? (T)w[base + lane] : (T)1;
          }
          row[k * P1] = v;
          for (int e = 1; e <= p; ++e) {
            v *= u;
            row[k * P1 + e] = v;
          }
        }
      } else {
        for (int e = 0; e < D * P1; ++e) row[e] = 0;
      }
    }
    __syncwarp();
    for (int j = 0; j < n; ++j) {
      const T* r0 = pw + j * D * P1;
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        if (t < nt) {
          const int o = qoff[t];
          T v = r0[o & 0xff] * r0[P1 + ((o >> 8) & 0xff)];
          if (D == 3) v *= r0[2 * P1 + (o >> 16)];
          acc[t] += v;
        }
      }
    }
  }
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int q = lane + 32 * t;
    if (t < nt && q < nfull) alpha[q] = acc[t] * inv_fact_t<T>(pd, q);
  }
  __syncwarp();
  compress_warp<T>(pd, alpha, s, lane);
  for (int q = lane; q < nj; q += 32) out[q] = (double)alpha[q];
}

template <int D, typename T, int NT>
__global__ void __launch_bounds__(32 * kP2mWarps) k_p2m_warp(
    PlanDev pd, const Geom* __restrict__ g, int L, int64_t nleaf, const int* __restrict__ start,
    const double* __restrict__ x0, const double* __restrict__ x1, const double* __restrict__ x2,
    const double* __restrict__ w, const float4* __restrict__ rel, double* __restrict__ mp) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t b = (int64_t)blockIdx.x * kP2mWarps + warp;
  if (b >= nleaf) return;
  const int nj = pd.nj;
  extern __shared__ __align__(16) unsigned char smraw[];
  const size_t per_warp = align_bytes<T>(sizeof(T) * (32 * D * (pd.p + 1) + pd.nfull));
  T* pw = reinterpret_cast<T*>(smraw + warp * per_warp);  // [32][D][p+1]
  T* alpha = pw + 32 * D * (pd.p + 1);                    // [nfull]
  const int i0 = start[b], i1 = start[b + 1];
  if (i0 == i1) {
    for (int q = lane; q < nj; q += 32) mp[(size_t)b * nj + q] = 0.0;
    return;
  }
  // the box-relative copy (float path) needs only the side: no FP64 centre
  int bc[3];
  double c[3] = {0.0, 0.0, 0.0}, s = g->s_leaf;
  if (!rel) box_center<D>(g, L, b, bc, c, &s);
  p2m_warp_body<D, T, NT>(pd, c, s, i0, i1, x0, x1, x2, w, rel, pw, alpha, lane,
                          mp + (size_t)b * nj);
}

// adaptive tree: one warp per leaf of level >= 2 with sources (FP64 inputs)
template <typename T, int NT>
__global__ void __launch_bounds__(32 * kP2mWarps) k_ap2m_warp(
    PlanDev pd, const Geom* __restrict__ g, ATree t, const double* __restrict__ x0,
    const double* __restrict__ x1, const double* __restrict__ x2, const double* __restrict__ w,
    double* __restrict__ mp) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = t.loff[2] + blockIdx.x * kP2mWarps + warp;
  if (b >= t.loff[t.maxlev + 1]) return;
  if (!t.leaf[b] || t.s1[b] == t.s0[b]) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  const size_t per_warp = align_bytes<T>(sizeof(T) * (32 * 3 * (pd.p + 1) + pd.nfull));
  T* pw = reinterpret_cast<T*>(smraw + warp * per_warp);
  T* alpha = pw + 32 * 3 * (pd.p + 1);
  int l, bc[3];
  abox(t, b, &l, bc);
  double c[3], s;
  abox_center(g, l, bc, c, &s);
  p2m_warp_body<3, T, NT>(pd, c, s, t.s0[b], t.s1[b], x0, x1, x2, w, nullptr, pw, alpha, lane,
                          mp + (size_t)b * pd.nj);
}

// ---------------------------------------------------------------------------
// M2M (Sec. 4.3, eqs. (mpole_translated_compressed_coeffs), (define_psi)):
// for each child, sigma_q = sum_{i <= q, i in j} h^{q-i}/(q-i)! beta_i with
// h = c_parent - c_child = +-s_child/2 per axis.  The multi-binomial shift is
// a product of 1D Taylor shifts, applied one axis at a time (x, then y on the
// embedded slabs m_s < c, then the slow axis into every slab); the children's
// sigmas are summed, rescaled to the parent's side (2^{-|q|}) and compressed
// once with the parent's recurrence (M^T is linear).  One block per parent.
// The children on either side of the centre along an axis have h = +1/2 and
// -1/2 (child units), so the shifts of a pair sum to
//   sum_t f_t (b0 + (-1)^t b1)[q - t],  f_t = (1/2)^t / t!:
// the pair's sum E and difference O are formed first and one shift reads E at
// even and O at odd t.  Summing right after each axis (linearity) leaves 4
// pairs for x, 2 for y and 1 for the slow axis.
// ---------------------------------------------------------------------------
__host__ __device__ inline size_t m2m_block_elems(int D, int nj, int nfull, int p) {
  return (size_t)((1 << D) + (1 << D) / 2 + (D == 3 ? 2 : 0)) * nj + nfull + p + 1;
}

// in place: (a, b) -> (a + b, a - b) for the n-element arrays a and b
template <typename T>
__device__ __forceinline__ void pair_eo(T* a, T* b, int n) {
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const T x = a[q], y = b[q];
    a[q] = x + y;
    b[q] = x - y;
  }
}

// body of M2M for a parent of side s: child ci's multipole is the row
// crow[ci] of mpc (-1: no child, taken as zero); the result goes to out
template <int D, typename T>
__device__ void m2m_body(const PlanDev& pd, double s, const int64_t* crow,
                         const double* __restrict__ mpc, double* __restrict__ out) {
  constexpr int NC = 1 << D;
  const int p = pd.p, c = pd.c, nfull = pd.nfull, nj = pd.nj;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* bet = reinterpret_cast<T*>(smraw);         // NC * nj: x pairs (E, O) of the children
  T* X = bet + NC * nj;                          // NC/2 * nj: x-shifted pairs, then y (E, O)
  T* Y = X + (NC / 2) * nj;                      // 2 * nj (D == 3): y-shifted, then slow (E, O)
  T* sig = Y + (D == 3 ? 2 * nj : 0);            // nfull
  T* f = sig + nfull;                            // p + 1: (1/2)^t / t!
  if (threadIdx.x <= p)  // the power of two is exact: one rounding in either type
    f[threadIdx.x] = pow2_neg<T>((int)threadIdx.x) * inv_fact_t<T>(pd, threadIdx.x);
  // children 2k and 2k+1 differ in the x bit: their sum and difference
  for (int e = threadIdx.x; e < (NC / 2) * nj; e += blockDim.x) {
    const int k = e / nj, q = e % nj;
    const T b0 = crow[2 * k] >= 0 ? (T)mpc[(size_t)crow[2 * k] * nj + q] : (T)0;
    const T b1 = crow[2 * k + 1] >= 0 ? (T)mpc[(size_t)crow[2 * k + 1] * nj + q] : (T)0;
    bet[2 * k * nj + q] = b0 + b1;
    bet[(2 * k + 1) * nj + q] = b0 - b1;
  }
  __syncthreads();
  // x shift of each pair on the stored slabs: X[k][q] = sum_{t <= q0} f_t (E|O)[q - t]
  for (int e = threadIdx.x; e < (NC / 2) * nj; e += blockDim.x) {
    const int k = e / nj, q = e % nj;
    const T* E = bet + 2 * k * nj;
    const T* O = E + nj;
    const int q0 = pd.mi[q].x;
    T ae = 0, ao = 0;
    int t = 0;
    for (; t + 1 <= q0; t += 2) {
      ae += f[t] * E[q - t];
      ao += f[t + 1] * O[q - t - 1];
    }
    if (t <= q0) ae += f[t] * E[q - t];
    X[e] = ae + ao;
  }
  __syncthreads();
  const T* Z = X;  // the slow axis' pair: E at 0, O at nj
  if (D == 3) {
    // X[2m], X[2m+1] differ in the y bit (slow bit m)
    pair_eo<T>(X, X + nj, nj);
    pair_eo<T>(X + 2 * nj, X + 3 * nj, nj);
    __syncthreads();
    for (int e = threadIdx.x; e < 2 * nj; e += blockDim.x) {
      const int m = e / nj, q = e % nj;
      const char4 mi = pd.mi[q];
      const T* E = X + 2 * m * nj;
      const T* O = E + nj;
      const int* fr = pd.frow + mi.z * (p + 1) + mi.y;  // row m_1 - t at fr[-t]
      T ae = 0, ao = 0;
      int t = 0;
      for (; t + 1 <= mi.y; t += 2) {
        ae += f[t] * E[fr[-t] + mi.x];
        ao += f[t + 1] * O[fr[-t - 1] + mi.x];
      }
      if (t <= mi.y) ae += f[t] * E[fr[-t] + mi.x];
      Y[e] = ae + ao;
    }
    __syncthreads();
    pair_eo<T>(Y, Y + nj, nj);
    Z = Y;
  } else {
    pair_eo<T>(X, X + nj, nj);  // X[0], X[1] differ in the slow bit
  }
  __syncthreads();
  // slow-axis shift into every slab, rescaled
  for (int q = threadIdx.x; q < nfull; q += blockDim.x) {
    const char4 m = pd.mi[q];
    const int q0 = m.x, q1 = D == 3 ? m.y : 0, qs = D == 3 ? m.z : m.y;
    T ae = 0, ao = 0;
    for (int is = 0; is <= min(qs, c - 1); ++is) {
      const int src = D == 3 ? pd.frow[is * (p + 1) + q1] + q0 : pd.frow[is] + q0;
      const int t = qs - is;
      if (t & 1) ao += f[t] * Z[nj + src];
      else ae += f[t] * Z[src];
    }
    sig[q] = (ae + ao) * pow2_neg<T>((int)m.w);
  }
  __syncthreads();
  compress_smem<T>(pd, sig, s);
  for (int q = threadIdx.x; q < nj; q += blockDim.x) out[q] = (double)sig[q];
}

template <int D, typename T>
__global__ void __launch_bounds__(kThreads) k_m2m(PlanDev pd, const Geom* __restrict__ g, int l,
                                                  const double* __restrict__ mpc,
                                                  double* __restrict__ mpp) {
  constexpr int NC = 1 << D;
  const int b = blockIdx.x;
  // box coordinates by integer arithmetic and the side alone (the centre is
  // not needed, and FP64 runs at 1/64 of the FP32 rate)
  const int nl = 1 << l, nlc = nl << 1;
  int bc[3] = {b & (nl - 1), (b >> l) & (nl - 1), D == 3 ? b >> (2 * l) : 0};
  const double s = __dmul_rn(g->size, pow2_neg<double>(l));
  int64_t crow[NC];
  for (int ci = 0; ci < NC; ++ci) {
    int64_t cb = 0;
    for (int k = D - 1; k >= 0; --k) cb = cb * nlc + (2 * bc[k] + ((ci >> k) & 1));
    crow[ci] = cb;
  }
  m2m_body<D, T>(pd, s, crow, mpc, mpp + (size_t)b * pd.nj);
}

// adaptive tree: one block per box of level l with children
template <typename T>
__global__ void __launch_bounds__(kThreads) k_am2m(PlanDev pd, const Geom* __restrict__ g,
                                                   ATree t, int l, double* __restrict__ mp) {
  const int b = t.loff[l] + blockIdx.x;
  if (t.leaf[b]) return;
  const double s = __dmul_rn(g->size, pow2_neg<double>(l));
  int64_t crow[8];
  for (int ci = 0; ci < 8; ++ci) crow[ci] = t.child[8 * b + ci];
  m2m_body<3, T>(pd, s, crow, mp, mp + (size_t)b * pd.nj);
}

// ---------------------------------------------------------------------------
// L2L (Sec. 4.2, eq. (l2l-expr), un-normalised): with Dt = M Lt_parent,
//   Lt_child_i += 2^{-|i|} sum_{q >= i} Dt_q (h/S)^{q-i} / (q-i)!,  i in j,
// h = c_child - c_parent = +-S/4 per axis.  Applied as 1D shifts along x, y
// and the slow axis (into the children's stored slabs).  The children on
// either side along an axis have h/S = -1/4 (bit 0) and +1/4 (bit 1): with
// g_t = (1/4)^t / t!, the even-t and odd-t partial sums se, so of one shift
// give se - so for bit 0 and se + so for bit 1, so each axis costs one shift
// per incoming array: 1 along x, 2 along y, 4 along the slow axis.
// ---------------------------------------------------------------------------
__host__ __device__ inline size_t l2l_block_elems(int D, int nfull, int p) {
  return (size_t)(D == 3 ? 7 : 3) * nfull + p + 1;
}

// body of L2L for a parent of side s with local row `par`: child ci receives
// into row crow[ci] of lcc (-1: no child)
template <int D, typename T>
__device__ void l2l_body(const PlanDev& pd, double s, const double* __restrict__ par,
                         const int64_t* crow, double* __restrict__ lcc) {
  constexpr int NC = 1 << D;
  const int p = pd.p, nfull = pd.nfull, nj = pd.nj;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Dt = reinterpret_cast<T*>(smraw);       // nfull
  T* X = Dt + nfull;                          // 2 * nfull: x bit 0, 1
  T* Y = X + 2 * nfull;                       // 4 * nfull (D == 3): sx + 2 sy
  T* g = Y + (D == 3 ? 4 * nfull : 0);        // p + 1: (1/4)^t / t!
  for (int q = threadIdx.x; q < nj; q += blockDim.x) Dt[q] = (T)par[q];
  if (threadIdx.x <= p)
    g[threadIdx.x] = pow2_neg<T>(2 * (int)threadIdx.x) * inv_fact_t<T>(pd, threadIdx.x);
  __syncthreads();
  decompress_smem<T>(pd, Dt, s);
  // x shift along the row of q: u[t] = Dt[q + t]
  for (int q = threadIdx.x; q < nfull; q += blockDim.x) {
    const char4 m = pd.mi[q];
    const int qs = D == 3 ? m.z : m.y, q1 = D == 3 ? m.y : 0;
    const int len = p - qs - q1 - m.x + 1;
    T se = 0, so = 0;
    int t = 0;
    for (; t + 1 < len; t += 2) {
      se += g[t] * Dt[q + t];
      so += g[t + 1] * Dt[q + t + 1];
    }
    if (t < len) se += g[t] * Dt[q + t];
    X[q] = se - so;
    X[nfull + q] = se + so;
  }
  __syncthreads();
  const T* Z = X;  // the slow axis' inputs: NC/2 arrays of nfull
  if (D == 3) {
    // y shift of each x variant: u[t] = X_sx[row m_1 + t]
    for (int e = threadIdx.x; e < 2 * nfull; e += blockDim.x) {
      const int sx = e / nfull, q = e % nfull;
      const char4 m = pd.mi[q];
      const T* Xv = X + sx * nfull;
      const int* fr = pd.frow + m.z * (p + 1) + m.y;
      const int len = p - m.z - m.x - m.y + 1;
      T se = 0, so = 0;
      int t = 0;
      for (; t + 1 < len; t += 2) {
        se += g[t] * Xv[fr[t] + m.x];
        so += g[t + 1] * Xv[fr[t + 1] + m.x];
      }
      if (t < len) se += g[t] * Xv[fr[t] + m.x];
      Y[sx * nfull + q] = se - so;        // sy = 0
      Y[(sx + 2) * nfull + q] = se + so;  // sy = 1
    }
    __syncthreads();
    Z = Y;
  }
  // slow axis into the stored slabs of the children (v, bit 0) and (v, bit 1)
  for (int e = threadIdx.x; e < (NC / 2) * nj; e += blockDim.x) {
    const int v = e / nj, i = e % nj;
    const int64_t r0 = crow[v], r1 = crow[v + NC / 2];
    if (r0 < 0 && r1 < 0) continue;
    const char4 m = pd.mi[i];
    const int i0 = m.x, i1 = D == 3 ? m.y : 0, is = D == 3 ? m.z : m.y;
    const T* Zv = Z + v * nfull;
    T se = 0, so = 0;
    for (int qs = is; qs <= p - i0 - i1; ++qs) {
      const int src = D == 3 ? pd.frow[qs * (p + 1) + i1] + i0 : pd.frow[qs] + i0;
      if ((qs - is) & 1) so += g[qs - is] * Zv[src];
      else se += g[qs - is] * Zv[src];
    }
    const T sc = pow2_neg<T>((int)m.w);
    if (r0 >= 0) lcc[(size_t)r0 * nj + i] += (double)((se - so) * sc);
    if (r1 >= 0) lcc[(size_t)r1 * nj + i] += (double)((se + so) * sc);
  }
}

template <int D, typename T>
__global__ void __launch_bounds__(kThreads) k_l2l(PlanDev pd, const Geom* __restrict__ g, int l,
                                                  const double* __restrict__ lcp,
                                                  double* __restrict__ lcc) {
  constexpr int NC = 1 << D;
  const int b = blockIdx.x;
  const int nl = 1 << l, nlc = nl << 1;  // integer box coordinates, the side alone
  int bc[3] = {b & (nl - 1), (b >> l) & (nl - 1), D == 3 ? b >> (2 * l) : 0};
  const double s = __dmul_rn(g->size, pow2_neg<double>(l));
  int64_t crow[NC];
  for (int ci = 0; ci < NC; ++ci) {
    int64_t cb = 0;
    for (int k = D - 1; k >= 0; --k) cb = cb * nlc + (2 * bc[k] + ((ci >> k) & 1));
    crow[ci] = cb;
  }
  l2l_body<D, T>(pd, s, lcp + (size_t)b * pd.nj, crow, lcc);
}

// adaptive tree: one block per box of level l (>= 2) with children and targets
template <typename T>
__global__ void __launch_bounds__(kThreads) k_al2l(PlanDev pd, const Geom* __restrict__ g,
                                                   ATree t, int l, double* __restrict__ lc) {
  const int b = t.loff[l] + blockIdx.x;
  if (t.leaf[b] || t.t1[b] == t.t0[b]) return;
  const double s = __dmul_rn(g->size, pow2_neg<double>(l));
  int64_t crow[8];
  for (int ci = 0; ci < 8; ++ci) {
    const int cb = t.child[8 * b + ci];
    crow[ci] = (cb >= 0 && t.t1[cb] > t.t0[cb]) ? cb : -1;
  }
  l2l_body<3, T>(pd, s, lc + (size_t)b * pd.nj, crow, lc);
}

}  // namespace

bool m2l_shared_tables(const fmm_plan_s* P) {
  const int prec = P->desc.precision;
  const bool tc = prec_tensor(prec);
  const bool fft = P->desc.m2l == FMM_M2L_FFT;
  return (tc || fft) && P->pd.d == 3 && kernel_homogeneous(P->pd.kernel);
}

// Residual of a PDE on the kernel's own derivatives (eq. (Pv): P applied to
// the derivatives of G vanishes when G satisfies the PDE).  The derivative
// table of one level is built for a root of side 4 (level-2 boxes of side 1)
// and read at the far offset h = (3, 2, 1) (2D: (3, 2)); for every m of slab
// 0 with |m| + c <= 2p the PDE's terms sum_t a_t d^{m + xi_t} G(h) must
// cancel.  Returns max |sum| / sum |terms| over those m, or -1 on a CUDA error.
double pde_residual(const PlanDev& pd, const std::vector<int>& hrow_host, int nterm,
                    const int* xi, const double* a) {
  const int D = pd.d, P2 = 2 * pd.p;
  const int noff = D == 3 ? 343 : 49;
  const int o = D == 3 ? (3 + 3) + 7 * (2 + 3) + 49 * (1 + 3) : (3 + 3) + 7 * (2 + 3);
  Geom g{};
  g.size = 4.0;
  void* dmem = nullptr;
  const size_t tab = sizeof(double) * (size_t)noff * pd.nh;
  if (cudaMalloc(&dmem, sizeof(Geom) + tab) != cudaSuccess) return -1.0;
  Geom* dg = static_cast<Geom*>(dmem);
  double* dh = reinterpret_cast<double*>(static_cast<char*>(dmem) + sizeof(Geom));
  std::vector<double> h(pd.nh);
  bool ok = cudaMemcpy(dg, &g, sizeof(Geom), cudaMemcpyHostToDevice) == cudaSuccess;
  const size_t smem = sizeof(double) * pd.nh * 2;
  if (ok && D == 3) {
    set_smem(k_deriv_tables<3>, smem);
    k_deriv_tables<3><<<noff, 128, smem>>>(pd, dg, dh);
  } else if (ok) {
    set_smem(k_deriv_tables<2>, smem);
    k_deriv_tables<2><<<noff, 128, smem>>>(pd, dg, dh);
  }
  ok = ok && cudaGetLastError() == cudaSuccess &&
       cudaMemcpy(h.data(), dh + (size_t)o * pd.nh, sizeof(double) * pd.nh,
                  cudaMemcpyDeviceToHost) == cudaSuccess;
  cudaFree(dmem);
  if (!ok) return -1.0;
  auto at = [&](int m0, int m1, int ms) {  // Hankel layout position (slabs 0..2c-2)
    return D == 3 ? hrow_host[(size_t)ms * (P2 + 1) + m1] + m0 : hrow_host[(size_t)ms] + m0;
  };
  // the scale of the derivatives of each total degree: a residual is
  // measured against it (an oscillating kernel's single derivative can be
  // near a zero, where its own size says nothing about the rounding)
  std::vector<double> dmax(P2 + 1, 0.0);
  for (int ms = 0; ms <= std::min(2 * pd.c - 2, P2); ++ms)
    for (int m1 = 0; m1 <= (D == 3 ? P2 - ms : 0); ++m1)
      for (int m0 = 0; m0 + m1 + ms <= P2; ++m0)
        dmax[m0 + m1 + ms] = std::max(dmax[m0 + m1 + ms], fabs(h[at(m0, m1, ms)]));
  double worst = 0.0;
  for (int deg = 0; deg + pd.c <= P2; ++deg)
    for (int m1 = 0; m1 <= (D == 3 ? deg : 0); ++m1) {
      const int m0 = deg - m1;
      double sum = 0.0, mag = 0.0;
      for (int t = 0; t < nterm; ++t) {
        const int* x = xi + 3 * t;
        const double v = a[t] * (D == 3 ? h[at(m0 + x[0], m1 + x[1], x[2])]
                                        : h[at(m0 + x[0], 0, x[1])]);
        sum += v;
        mag += fabs(a[t]) * dmax[deg + x[0] + x[1] + x[2]];
      }
      if (mag > 0.0) worst = std::max(worst, fabs(sum) / mag);
    }
  return worst;
}

cudaError_t launch_deriv_tables(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st,
                                int* nl) {
  const PlanDev& pd = P->pd;
  const int L = P->desc.levels;
  const size_t smem = sizeof(double) * pd.nh * 2;
  // the tensor-core and FFT forms of M2L read only level 2's table for a
  // homogeneous kernel
  // adaptive plans: levels 2..deepest level of the current tree
  const int nlev = L < 0 ? P->deriv_levels - 1 : (m2l_shared_tables(P) ? 1 : L - 1);
  if (pd.d == 3) {
    set_smem(k_deriv_tables<3>, smem);
    k_deriv_tables<3><<<nlev * 343, 128, smem, st>>>(pd, ws.geom, ws.htab);
  } else {
    set_smem(k_deriv_tables<2>, smem);
    k_deriv_tables<2><<<(L - 1) * 49, 128, smem, st>>>(pd, ws.geom, ws.htab);
  }
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_p2m(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st, int* nl) {
  const PlanDev& pd = P->pd;
  const int L = P->desc.levels, d = pd.d;
  const int64_t nleaf = nbox_at(d, L);
  const bool f64 = P->desc.precision == FMM_PREC_FP64;
  if (!f64 && launch_p2m_f32(P, ws, st)) {  // 3D, box-relative float points
    ++*nl;
    return cudaGetLastError();
  }
  const size_t tsz = f64 ? 8 : 4;
  const size_t smem = align_bytes<double>(tsz * 32 * d * (pd.p + 1)) + tsz * pd.nfull;
  double* mpL = ws.mp + ws.lev_off[L] * pd.nj;
  if (pd.nfull <= 32 * kWarpTerms) {
    const size_t tsz2 = f64 ? 8 : 4;
    const size_t pwb = align_bytes<double>(tsz2 * (32 * d * (pd.p + 1) + pd.nfull));
    const size_t sm2 = pwb * kP2mWarps;
    const unsigned nb = (unsigned)((nleaf + kP2mWarps - 1) / kP2mWarps);
    const int ntl = (pd.nfull + 31) / 32;
#define P2MW_NT(DD, TT, NTT)                                                                \
  do {                                                                                      \
    set_smem(k_p2m_warp<DD, TT, NTT>, sm2);                                                 \
    k_p2m_warp<DD, TT, NTT><<<nb, 32 * kP2mWarps, sm2, st>>>(                               \
        pd, ws.geom, L, nleaf, ws.sstart, ws.sx[0], ws.sx[1], ws.sx[2], ws.sw, ws.sxr, mpL); \
  } while (0)
#define P2MW(DD, TT)                                                                        \
  do {                                                                                      \
    if (ntl <= 4) P2MW_NT(DD, TT, 4);                                                       \
    else if (ntl <= 10) P2MW_NT(DD, TT, 10);                                                \
    else if (ntl <= 16) P2MW_NT(DD, TT, 16);                                                \
    else P2MW_NT(DD, TT, 32);                                                               \
  } while (0)
    if (d == 3) {
      if (f64) P2MW(3, double); else P2MW(3, float);
    } else {
      if (f64) P2MW(2, double); else P2MW(2, float);
    }
#undef P2MW
#undef P2MW_NT
    ++*nl;
    return cudaGetLastError();
  }
#define P2M_LAUNCH(DD, TT)                                                                  \
  do {                                                                                      \
    set_smem(k_p2m<DD, TT>, smem);                                                          \
    k_p2m<DD, TT><<<(unsigned)nleaf, kThreads, smem, st>>>(pd, ws.geom, L, ws.sstart,       \
                                                           ws.sx[0], ws.sx[1], ws.sx[2],    \
                                                           ws.sw, ws.sxr, mpL);             \
  } while (0)
  if (d == 3) {
    if (f64) P2M_LAUNCH(3, double); else P2M_LAUNCH(3, float);
  } else {
    if (f64) P2M_LAUNCH(2, double); else P2M_LAUNCH(2, float);
  }
#undef P2M_LAUNCH
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_m2m(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st, int* nl) {
  const PlanDev& pd = P->pd;
  const int L = P->desc.levels, d = pd.d;
  // In the mixed modes the leaf multipoles come from the float P2M, so their
  // first shift runs in float too; shifts higher in the tree keep FP64-class
  // precision in double-word floats (FP64 in the FP64 mode).
  const bool mixed = P->desc.precision != FMM_PREC_FP64;
  if (d == 3 && passes_f32_order(pd.p)) {  // warp-per-box kernels
    for (int l = L - 1; l >= 2; --l) {
      launch_m2m_warp(P, ws, l, !mixed ? kShiftF64 : l == L - 1 ? kShiftF32 : kShiftDW, st);
      ++*nl;
    }
    return cudaGetLastError();
  }
  for (int l = L - 1; l >= 2; --l) {
    const double* mpc = ws.mp + ws.lev_off[l + 1] * pd.nj;
    double* mpp = ws.mp + ws.lev_off[l] * pd.nj;
    const bool f32 = mixed && l == L - 1;
    const size_t tsz = f32 ? 4 : 8;  // sizeof(dwf) == sizeof(double)
    const size_t smem = tsz * m2m_block_elems(d, pd.nj, pd.nfull, pd.p);
#define M2M_GO(DD, TT)                                                                     \
  do {                                                                                     \
    set_smem(k_m2m<DD, TT>, smem);                                                         \
    k_m2m<DD, TT><<<(unsigned)nbox_at(DD, l), kThreads, smem, st>>>(pd, ws.geom, l, mpc, mpp); \
  } while (0)
    if (d == 3) {
      if (f32) M2M_GO(3, float); else if (mixed) M2M_GO(3, dwf); else M2M_GO(3, double);
    } else {
      if (f32) M2M_GO(2, float); else if (mixed) M2M_GO(2, dwf); else M2M_GO(2, double);
    }
#undef M2M_GO
    ++*nl;
  }
  return cudaGetLastError();
}

cudaError_t launch_l2l(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st, int* nl) {
  const PlanDev& pd = P->pd;
  const int L = P->desc.levels, d = pd.d;
  // In the mixed modes the leaf locals feed the float L2P, so the last shift
  // (to the leaves) runs in float; shifts higher in the tree keep FP64-class
  // precision in double-word floats (FP64 in the FP64 mode).
  const bool mixed = P->desc.precision != FMM_PREC_FP64;
  if (d == 3 && passes_f32_order(pd.p)) {  // warp-per-box kernels
    for (int l = 2; l < L; ++l) {
      launch_l2l_warp(P, ws, l, !mixed ? kShiftF64 : l == L - 1 ? kShiftF32 : kShiftDW, st);
      ++*nl;
    }
    return cudaGetLastError();
  }
  for (int l = 2; l < L; ++l) {
    const double* lcp = ws.lc + ws.lev_off[l] * pd.nj;
    double* lcc = ws.lc + ws.lev_off[l + 1] * pd.nj;
    const bool f32 = mixed && l == L - 1;
    const size_t tsz = f32 ? 4 : 8;  // sizeof(dwf) == sizeof(double)
    const size_t smem = tsz * l2l_block_elems(d, pd.nfull, pd.p);
#define L2L_GO(DD, TT)                                                                     \
  do {                                                                                     \
    set_smem(k_l2l<DD, TT>, smem);                                                         \
    k_l2l<DD, TT><<<(unsigned)nbox_at(DD, l), kThreads, smem, st>>>(pd, ws.geom, l, lcp, lcc); \
  } while (0)
    if (d == 3) {
      if (f32) L2L_GO(3, float); else if (mixed) L2L_GO(3, dwf); else L2L_GO(3, double);
    } else {
      if (f32) L2L_GO(2, float); else if (mixed) L2L_GO(2, dwf); else L2L_GO(2, double);
    }
#undef L2L_GO
    ++*nl;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Adaptive tree: P2L over X (eq. (stored_local_coeffs)) into every box of
// level >= 2 that holds more than |j| targets (below that the leaves sum the
// X leaves' sources directly, which costs less).  X(B) = the leaves coarser than B that are
// adjacent to P(B) but not to B; each is a neighbour of B's ancestor at its
// own level, so the block walks the 27 neighbours of every ancestor.  Threads
// share the sources of each X leaf; every source adds w * Ht((c_B - y)/s)
// to the box's local expansion (shared-memory atomics).
// ---------------------------------------------------------------------------
namespace {

constexpr int kAThreads = 64;

__global__ void __launch_bounds__(kAThreads) k_ap2l(PlanDev pd, const Geom* __restrict__ g,
                                                    ATree t, const double* __restrict__ sx0,
                                                    const double* __restrict__ sx1,
                                                    const double* __restrict__ sx2,
                                                    const double* __restrict__ sw,
                                                    double* __restrict__ lc) {
  const int b = t.loff[2] + blockIdx.x;
  // a box of at most |j| targets has its X pairs summed directly by the leaves
  if (b >= t.loff[t.maxlev + 1] || t.t1[b] - t.t0[b] <= pd.nj) return;
  const int nj = pd.nj;
  int l, bc[3];
  abox(t, b, &l, bc);
  double cb[3], s;
  abox_center(g, l, bc, cb, &s);
  extern __shared__ __align__(16) double smd[];
  double* Lacc = smd;
  const int sl = min(pd.c, pd.p + 1) * (pd.p + 1);
  const int per = (kernel_screened(pd.kernel) ? 6 : 3) * sl;
  double* S = smd + ((nj + 1) & ~1) + threadIdx.x * per;
  for (int i = threadIdx.x; i < nj; i += blockDim.x) Lacc[i] = 0.0;
  __syncthreads();
  const double inv_s = 1.0 / s, lam = pd.lam * s, scale = deriv_scale(pd, s);
  const int pc[3] = {bc[0] >> 1, bc[1] >> 1, bc[2] >> 1};
  bool any = false;
  for (int lp = l - 1; lp >= 0; --lp) {
    const int a[3] = {bc[0] >> (l - lp), bc[1] >> (l - lp), bc[2] >> (l - lp)};
    for (int nb = 0; nb < 27; ++nb) {
      const int nc[3] = {a[0] + nb % 3 - 1, a[1] + (nb / 3) % 3 - 1, a[2] + nb / 9 - 1};
      const int A = alookup(t, lp, nc);
      if (A < 0 || !t.leaf[A]) continue;
      if (!aadjacent(lp, nc, l - 1, pc) || aadjacent(lp, nc, l, bc)) continue;
      any = true;
      for (int q = t.s0[A] + threadIdx.x; q < t.s1[A]; q += blockDim.x) {
        const double x[3] = {(cb[0] - sx0[q]) * inv_s, (cb[1] - sx1[q]) * inv_s,
                             (cb[2] - sx2[q]) * inv_s};
        deriv_point(pd, x, lam, scale * sw[q], S, sl,
                    [&](int pos, double v) { atomicAdd(&Lacc[pos], v); });
      }
    }
  }
  if (!any) return;  // block-uniform
  __syncthreads();
  for (int i = threadIdx.x; i < nj; i += blockDim.x) lc[(size_t)b * nj + i] += Lacc[i];
}

// Float form of k_ap2l (mixed-precision modes): the X leaf's sources are
// staged as float (c_B - y)/s_B (from the float pairs of the sources and of
// the centre: no FP64 arithmetic per source), each
// thread runs the float derivative recurrence for its sources and adds
// w * Ht into a float accumulator in shared memory.
constexpr int kAFStage = 256;

__global__ void __launch_bounds__(kAThreads) k_ap2l_f32(PlanDev pd, const Geom* __restrict__ g,
                                                        ATree t, const float4* __restrict__ sxh,
                                                        const float4* __restrict__ sxl,
                                                        double* __restrict__ lc) {
  const int b = t.loff[2] + blockIdx.x;
  // a box of at most |j| targets has its X pairs summed directly by the leaves
  if (b >= t.loff[t.maxlev + 1] || t.t1[b] - t.t0[b] <= pd.nj) return;
  const int nj = pd.nj;
  int l, bc[3];
  abox(t, b, &l, bc);
  double cb[3], s;
  abox_center(g, l, bc, cb, &s);
  extern __shared__ __align__(16) float smp[];
  float4* stage = reinterpret_cast<float4*>(smp);  // kAFStage
  float* Lacc = smp + 4 * kAFStage;
  const int sl = min(pd.c, pd.p + 1) * (pd.p + 1);
  const int per = (kernel_screened(pd.kernel) ? 6 : 3) * sl;
  float* S = Lacc + ((nj + 3) & ~3) + threadIdx.x * per;
  for (int i = threadIdx.x; i < nj; i += blockDim.x) Lacc[i] = 0.f;
  const double inv_s = 1.0 / s;
  const float ch[3] = {(float)cb[0], (float)cb[1], (float)cb[2]};
  const float cl[3] = {(float)(cb[0] - (double)ch[0]), (float)(cb[1] - (double)ch[1]),
                       (float)(cb[2] - (double)ch[2])};
  const float inv_sf = (float)inv_s;
  const float lam = (float)(pd.lam * s), scale = (float)deriv_scale(pd, s);
  const int pc[3] = {bc[0] >> 1, bc[1] >> 1, bc[2] >> 1};
  bool any = false;
  for (int lp = l - 1; lp >= 0; --lp) {
    const int an[3] = {bc[0] >> (l - lp), bc[1] >> (l - lp), bc[2] >> (l - lp)};
    for (int nb = 0; nb < 27; ++nb) {
      const int nc[3] = {an[0] + nb % 3 - 1, an[1] + (nb / 3) % 3 - 1, an[2] + nb / 9 - 1};
      const int A = alookup(t, lp, nc);
      if (A < 0 || !t.leaf[A]) continue;
      if (!aadjacent(lp, nc, l - 1, pc) || aadjacent(lp, nc, l, bc)) continue;
      any = true;
      for (int jb = t.s0[A]; jb < t.s1[A]; jb += kAFStage) {
        const int n = min(kAFStage, t.s1[A] - jb);
        __syncthreads();
        for (int q = threadIdx.x; q < n; q += blockDim.x) {
          const float4 h = sxh[jb + q], o = sxl[jb + q];
          stage[q] = make_float4(__fmul_rn(__fadd_rn(ch[0] - h.x, cl[0] - o.x), inv_sf),
                                 __fmul_rn(__fadd_rn(ch[1] - h.y, cl[1] - o.y), inv_sf),
                                 __fmul_rn(__fadd_rn(ch[2] - h.z, cl[2] - o.z), inv_sf), h.w);
        }
        __syncthreads();
        // A warp takes 32 sources at a time (lanes past the end take a
        // weightless point), so every lane emits the same coefficient at the
        // same step: the warp sums it with shuffles and one lane adds it, in
        // place of 32 shared-memory atomics on one address.
        const int lane = threadIdx.x & 31;
        for (int q0 = threadIdx.x & ~31; q0 < n; q0 += blockDim.x) {  // warp-uniform
          const int q = q0 + lane;
          const float4 v = q < n ? stage[q] : make_float4(4.f, 4.f, 4.f, 0.f);
          const float x[3] = {v.x, v.y, v.z};
          deriv_point<float>(pd, x, lam, scale * v.w, S, sl, [&](int pos, float h) {
            for (int off = 16; off > 0; off >>= 1) h += __shfl_xor_sync(0xffffffffu, h, off);
            if (lane == 0) atomicAdd(&Lacc[pos], h);
          });
        }
      }
    }
  }
  if (!any) return;  // block-uniform
  __syncthreads();
  for (int i = threadIdx.x; i < nj; i += blockDim.x) lc[(size_t)b * nj + i] += (double)Lacc[i];
}

}  // namespace

cudaError_t launch_adaptive_upward(const fmm_plan_s* P, const Workspace& ws, const ATree& t,
                                   cudaStream_t st, int* nl) {
  const PlanDev& pd = P->pd;
  const int nbox = t.loff[t.maxlev + 1];
  if (t.maxlev < 2) return cudaGetLastError();
  // P2M at the leaves of level >= 2 (warp per leaf)
  {
    const int n = nbox - t.loff[2];
    const size_t pwb = align_bytes<double>(sizeof(double) * (32 * 3 * (pd.p + 1) + pd.nfull));
    const size_t sm2 = pwb * kP2mWarps;
    const unsigned nb = (unsigned)((n + kP2mWarps - 1) / kP2mWarps);
    const int ntl = (pd.nfull + 31) / 32;
#define AP2M(TT, NTT)                                                                      \
  do {                                                                                     \
    set_smem(k_ap2m_warp<TT, NTT>, sm2);                                                   \
    k_ap2m_warp<TT, NTT><<<nb, 32 * kP2mWarps, sm2, st>>>(pd, ws.geom, t, ws.sx[0],        \
                                                          ws.sx[1], ws.sx[2], ws.sw, ws.mp); \
  } while (0)
#define AP2MN(TT)                                                                          \
  do {                                                                                     \
    if (ntl <= 4) AP2M(TT, 4);                                                             \
    else if (ntl <= 10) AP2M(TT, 10);                                                      \
    else if (ntl <= 16) AP2M(TT, 16);                                                      \
    else AP2M(TT, 32);                                                                     \
  } while (0)
    if (P->desc.precision == FMM_PREC_FP64) AP2MN(double);
    else if (!launch_ap2m_f32(P, ws, t, st)) AP2MN(float);  // float sums from FP64 inputs
#undef AP2MN
#undef AP2M
    ++*nl;
  }
  // M2M, deepest parents first: FP64, or double-word floats in the mixed modes
  const bool f64 = P->desc.precision == FMM_PREC_FP64;
  const size_t smem = sizeof(double) * m2m_block_elems(3, pd.nj, pd.nfull, pd.p);
  if (f64) set_smem(k_am2m<double>, smem);
  else set_smem(k_am2m<dwf>, smem);
  for (int l = t.maxlev - 1; l >= 2; --l) {
    const int n = t.loff[l + 1] - t.loff[l];
    if (f64) k_am2m<double><<<(unsigned)n, kThreads, smem, st>>>(pd, ws.geom, t, l, ws.mp);
    else k_am2m<dwf><<<(unsigned)n, kThreads, smem, st>>>(pd, ws.geom, t, l, ws.mp);
    ++*nl;
  }
  return cudaGetLastError();
}

cudaError_t launch_adaptive_p2l_l2l(const fmm_plan_s* P, const Workspace& ws, const ATree& t,
                                    cudaStream_t st, int* nl) {
  const PlanDev& pd = P->pd;
  if (t.maxlev < 2) return cudaGetLastError();
  const int nbox = t.loff[t.maxlev + 1];
  {
    const int sl = std::min(pd.c, pd.p + 1) * (pd.p + 1);
    const int per = (kernel_screened(pd.kernel) ? 6 : 3) * sl;
    if (P->desc.precision == FMM_PREC_FP64) {
      const size_t smem = sizeof(double) * (((pd.nj + 1) & ~1) + (size_t)per * kAThreads);
      set_smem(k_ap2l, smem);
      k_ap2l<<<(unsigned)(nbox - t.loff[2]), kAThreads, smem, st>>>(
          pd, ws.geom, t, ws.sx[0], ws.sx[1], ws.sx[2], ws.sw, ws.lc);
    } else {
      const size_t smem =
          sizeof(float) * (4 * kAFStage + ((pd.nj + 3) & ~3) + (size_t)per * kAThreads);
      set_smem(k_ap2l_f32, smem);
      k_ap2l_f32<<<(unsigned)(nbox - t.loff[2]), kAThreads, smem, st>>>(pd, ws.geom, t, ws.asxh,
                                                                        ws.asxl, ws.lc);
    }
    ++*nl;
  }
  // L2L: FP64, or double-word floats in the mixed modes
  const bool f64 = P->desc.precision == FMM_PREC_FP64;
  const size_t smem = sizeof(double) * l2l_block_elems(3, pd.nfull, pd.p);
  if (f64) set_smem(k_al2l<double>, smem);
  else set_smem(k_al2l<dwf>, smem);
  for (int l = 2; l < t.maxlev; ++l) {
    const int n = t.loff[l + 1] - t.loff[l];
    if (f64) k_al2l<double><<<(unsigned)n, kThreads, smem, st>>>(pd, ws.geom, t, l, ws.lc);
    else k_al2l<dwf><<<(unsigned)n, kThreads, smem, st>>>(pd, ws.geom, t, l, ws.lc);
    ++*nl;
  }
  return cudaGetLastError();
}
