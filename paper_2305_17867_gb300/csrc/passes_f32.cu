// Float kernels of the upward and downward passes of 3D uniform trees in the
// mixed-precision modes, one warp per box.  The expansions stay FP64 in
// memory; every step in between runs in float, so that no FP64 instruction
// (1/64 of the FP32 rate on this GPU) sits on the path.
//
//  * P2M (Sec. 3.4): alpha_m = sum_y w ((c - y)/s)^m / m!, then beta = M^T alpha.
//    The monomials of one source come in segments of up to four consecutive
//    m_0 of a row (m_1, m_s) of the full layout: the first from per-source
//    power tables, the others by repeated multiplication with x.  Each lane
//    owns two segments; two sources share every instruction (f32x2).
//  * M2M (Sec. 4.3, eq. (mpole_translated_compressed_coeffs)) and L2L
//    (Sec. 4.2, eq. (l2l-expr)): the multi-index Taylor shift is a product of
//    1D shifts along x, y and the slow axis.  A lane holds one row (column,
//    pillar) of coefficients in registers and applies the 1D shift with the
//    coefficients h^t / t! as compile-time constants.  The children on either
//    side of the parent's centre differ in the sign of h only: the even and
//    odd powers are summed apart and their sum and difference serve both.
//    M2M sums the children before the next axis (the shift is linear), so the
//    y shift runs on 4 and the slow-axis shift on 2 arrays instead of 8.
//  * L2P (eq. (stored_local_coeffs) at the targets): nested Horner in x, y
//    and the slow axis over the decompressed Lt_m / m!, with the gradient by
//    the derivative recurrence of Horner's scheme.  A warp takes four leaves;
//    their targets run as one list over the lanes.
//
// Orders p in {4, 6, 8, 10, 12, 16} are compiled (the register rows are
// sized by p); other orders keep the block-per-box kernels.
#include "adaptive.cuh"
#include "expansions.cuh"
#include "f32x2.cuh"
#include "passes_f32.cuh"

namespace {

// ---------------------------------------------------------------------------
// Taylor shift coefficients h^t / t! for h = 1/2 (M2M: child centre to
// parent centre in child units) and h = 1/4 (L2L: parent centre to child
// centre in parent units), t = 0..20.
// ---------------------------------------------------------------------------
constexpr double taylor_coef(int t, double h) {
  double v = 1.0;
  for (int k = 1; k <= t; ++k) v *= h / k;
  return v;
}
#define TC21(h)                                                                           \
  {(float)taylor_coef(0, h),  (float)taylor_coef(1, h),  (float)taylor_coef(2, h),        \
   (float)taylor_coef(3, h),  (float)taylor_coef(4, h),  (float)taylor_coef(5, h),        \
   (float)taylor_coef(6, h),  (float)taylor_coef(7, h),  (float)taylor_coef(8, h),        \
   (float)taylor_coef(9, h),  (float)taylor_coef(10, h), (float)taylor_coef(11, h),       \
   (float)taylor_coef(12, h), (float)taylor_coef(13, h), (float)taylor_coef(14, h),       \
   (float)taylor_coef(15, h), (float)taylor_coef(16, h), (float)taylor_coef(17, h),       \
   (float)taylor_coef(18, h), (float)taylor_coef(19, h), (float)taylor_coef(20, h)}
__constant__ float c_half[FMM_MAXP + 1] = TC21(0.5);
__constant__ float c_quarter[FMM_MAXP + 1] = TC21(0.25);
#undef TC21
#define TD21(h)                                                                           \
  {taylor_coef(0, h),  taylor_coef(1, h),  taylor_coef(2, h),  taylor_coef(3, h),         \
   taylor_coef(4, h),  taylor_coef(5, h),  taylor_coef(6, h),  taylor_coef(7, h),         \
   taylor_coef(8, h),  taylor_coef(9, h),  taylor_coef(10, h), taylor_coef(11, h),        \
   taylor_coef(12, h), taylor_coef(13, h), taylor_coef(14, h), taylor_coef(15, h),        \
   taylor_coef(16, h), taylor_coef(17, h), taylor_coef(18, h), taylor_coef(19, h),        \
   taylor_coef(20, h)}
__constant__ double c_half_d[FMM_MAXP + 1] = TD21(0.5);
__constant__ double c_quarter_d[FMM_MAXP + 1] = TD21(0.25);
#undef TD21
// the same as double-word floats: (float) v and (float) (v - (float) v)
constexpr float2 dw_split(double v) {
  return float2{(float)v, (float)(v - (double)(float)v)};
}
#define TW21(h)                                                                           \
  {dw_split(taylor_coef(0, h)),  dw_split(taylor_coef(1, h)),  dw_split(taylor_coef(2, h)),  \
   dw_split(taylor_coef(3, h)),  dw_split(taylor_coef(4, h)),  dw_split(taylor_coef(5, h)),  \
   dw_split(taylor_coef(6, h)),  dw_split(taylor_coef(7, h)),  dw_split(taylor_coef(8, h)),  \
   dw_split(taylor_coef(9, h)),  dw_split(taylor_coef(10, h)), dw_split(taylor_coef(11, h)), \
   dw_split(taylor_coef(12, h)), dw_split(taylor_coef(13, h)), dw_split(taylor_coef(14, h)), \
   dw_split(taylor_coef(15, h)), dw_split(taylor_coef(16, h)), dw_split(taylor_coef(17, h)), \
   dw_split(taylor_coef(18, h)), dw_split(taylor_coef(19, h)), dw_split(taylor_coef(20, h))}
__constant__ float2 c_half_w[FMM_MAXP + 1] = TW21(0.5);
__constant__ float2 c_quarter_w[FMM_MAXP + 1] = TW21(0.25);
#undef TW21

// h^t / t! in the kernel's arithmetic (H = 0: h = 1/2, H = 1: h = 1/4)
template <typename T, int H>
__device__ __forceinline__ T shift_coef(int t);
template <>
__device__ __forceinline__ float shift_coef<float, 0>(int t) { return c_half[t]; }
template <>
__device__ __forceinline__ float shift_coef<float, 1>(int t) { return c_quarter[t]; }
template <>
__device__ __forceinline__ double shift_coef<double, 0>(int t) { return c_half_d[t]; }
template <>
__device__ __forceinline__ double shift_coef<double, 1>(int t) { return c_quarter_d[t]; }
template <>
__device__ __forceinline__ dwf shift_coef<dwf, 0>(int t) { return dwf(c_half_w[t].x, c_half_w[t].y); }
template <>
__device__ __forceinline__ dwf shift_coef<dwf, 1>(int t) {
  return dwf(c_quarter_w[t].x, c_quarter_w[t].y);
}

constexpr int kWarps = 8;  // boxes (warps) per block, fewer when shared memory is short

// Position of (m_0 = a, m_1, m_s) in the full layout of order P1 - 1: slabs
// by m_s (slab k holds (P1-k)(P1-k+1)/2 entries, so slabs 0..m_s-1 hold the
// tetrahedral difference T(P1) - T(P1 - m_s), T(n) = n(n+1)(n+2)/6), rows by
// m_1 inside a slab, m_0 contiguous.  The stored set is the prefix m_s < c.
template <int P1>
__device__ __forceinline__ int fpos(int ms, int m1, int a) {
  const int n = P1 - ms;
  return (P1 * (P1 + 1) * (P1 + 2) - n * (n + 1) * (n + 2)) / 6 + m1 * n - m1 * (m1 - 1) / 2 + a;
}

// The r-th pair (i, k) with k <= P1 - 1 - i in i-major order: rows (m_s, m_1)
// of the full layout, columns (m_s, m_0), or pillars (m_1, m_0).
template <int P1>
__device__ __forceinline__ void pair_of(int r, int& i, int& k) {
  int s = 0, base = 0;
  while (r >= base + (P1 - s)) {
    base += P1 - s;
    ++s;
  }
  i = s;
  k = r - base;
}

// ---------------------------------------------------------------------------
// M2M.  Upward 1D shift of the two children on either side along one axis,
// summed: out[k] = sum_{t<=k} f_t (u0[k-t] + (-1)^t u1[k-t]), f_t = (1/2)^t/t!
// (child bit 0 lies below the parent's centre, h = +1/2; bit 1 above, -1/2).
// pos(k) gives the k-th position along the line, len its length.
// ---------------------------------------------------------------------------
template <typename T, int P1, typename Pos>
__device__ __forceinline__ void shift_up_pair(const T* __restrict__ u0, const T* __restrict__ u1,
                                              int len, Pos pos, T* __restrict__ out) {
  T e[P1], o[P1];
#pragma unroll
  for (int k = 0; k < P1; ++k) {
    T a0 = 0, a1 = 0;
    if (k < len) {
      const int q = pos(k);
      a0 = u0[q];
      a1 = u1[q];
    }
    e[k] = a0 + a1;
    o[k] = a0 - a1;
  }
#pragma unroll
  for (int k = 0; k < P1; ++k) {
    T acc = 0;
#pragma unroll
    for (int t = 0; t <= k; ++t) acc = fma(shift_coef<T, 0>(t), (t & 1) ? o[k - t] : e[k - t], acc);
    if (k < len) out[pos(k)] = acc;
  }
}

__host__ __device__ inline int m2m_elems(int nj, int nfull) {
  return (14 * nj + nfull + 3) & ~3;  // 8 children, 4 + 2 partial sums, the full sigma
}

template <typename T, int P>
__global__ void __launch_bounds__(32 * kWarps) k_m2m_w(PlanDev pd, const Geom* __restrict__ g,
                                                       int l, const double* __restrict__ mpc,
                                                       double* __restrict__ mpp) {
  constexpr int P1 = P + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nl = 1 << l;
  const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (b >= (int64_t)nl * nl * nl) return;
  const int c = min(pd.c, P1), nj = pd.nj;
  extern __shared__ __align__(16) unsigned char smw[];
  T* B = reinterpret_cast<T*>(smw) + (size_t)warp * m2m_elems(nj, pd.nfull);  // [8][nj] children
  T* X = B + 8 * nj;                                                          // [4][nj] (sy + 2 sz)
  T* Y = X + 4 * nj;                                                          // [2][nj] (sz)
  T* S = Y + 2 * nj;                                                          // [nfull] sigma
  const int bx = (int)(b & (nl - 1)), by = (int)((b >> l) & (nl - 1)), bz = (int)(b >> (2 * l));
  const int64_t nlc = 2 * (int64_t)nl;
  for (int ci = 0; ci < 8; ++ci) {
    const int64_t cb =
        ((2 * bz + (ci >> 2)) * nlc + (2 * by + ((ci >> 1) & 1))) * nlc + (2 * bx + (ci & 1));
    const double* src = mpc + cb * nj;
    T* dst = B + ci * nj;
    for (int q = lane; q < nj; q += 32) dst[q] = (T)src[q];
  }
  __syncwarp();
  const int nrs = c * P1 - c * (c - 1) / 2;  // rows (m_1, m_s < c) of the stored set
  // x: rows of children 2v and 2v + 1 (x bits 0, 1), v = sy + 2 sz
  for (int v = 0; v < 4; ++v)
    for (int r = lane; r < nrs; r += 32) {
      int ms, m1;
      pair_of<P1>(r, ms, m1);
      const int st = fpos<P1>(ms, m1, 0);
      shift_up_pair<T, P1>(B + 2 * v * nj + st, B + (2 * v + 1) * nj + st, P1 - ms - m1,
                           [](int k) { return k; }, X + v * nj + st);
    }
  __syncwarp();
  // y: columns (m_s < c, m_0) of the sums with y bits 0, 1
  for (int sz = 0; sz < 2; ++sz)
    for (int r = lane; r < nrs; r += 32) {
      int ms, a;
      pair_of<P1>(r, ms, a);
      shift_up_pair<T, P1>(X + 2 * sz * nj, X + (2 * sz + 1) * nj, P1 - ms - a,
                           [&](int k) { return fpos<P1>(ms, k, a); }, Y + sz * nj);
    }
  __syncwarp();
  // slow axis: pillars (m_1, m_0) from the stored slabs into every slab,
  // rescaled to the parent's side (2^-|q|)
  constexpr int NPIL = P1 * (P1 + 1) / 2;
  for (int r = lane; r < NPIL; r += 32) {
    int m1, a;
    pair_of<P1>(r, m1, a);
    const int len = P1 - m1 - a, cc = min(c, len);
    T e[P1], o[P1];
#pragma unroll
    for (int is = 0; is < P1; ++is) {
      T a0 = 0, a1 = 0;
      if (is < cc) {
        const int q = fpos<P1>(is, m1, a);
        a0 = Y[q];
        a1 = Y[nj + q];
      }
      e[is] = a0 + a1;
      o[is] = a0 - a1;
    }
#pragma unroll
    for (int qs = 0; qs < P1; ++qs) {
      T acc = 0;
#pragma unroll
      for (int is = 0; is <= qs; ++is)
        acc = fma(shift_coef<T, 0>(qs - is), ((qs - is) & 1) ? o[is] : e[is], acc);
      if (qs < len) S[fpos<P1>(qs, m1, a)] = acc * pow2_neg<T>(a + m1 + qs);
    }
  }
  __syncwarp();
  compress_warp<T>(pd, S, __dmul_rn(g->size, pow2_neg<double>(l)), lane);
  double* out = mpp + b * nj;
  for (int q = lane; q < nj; q += 32) out[q] = (double)S[q];
}

// ---------------------------------------------------------------------------
// L2L.  Downward 1D shift along one axis in both directions:
//   se[k] = sum_{t even} g_t u[k+t],  so[k] = sum_{t odd} g_t u[k+t],
// g_t = (1/4)^t / t!; the child below the centre (bit 0, h/S = -1/4) gets
// se - so, the one above (bit 1, +1/4) se + so.
// ---------------------------------------------------------------------------
template <typename T, int P1, typename Pos>
__device__ __forceinline__ void shift_down_pair(const T* __restrict__ u, int len, Pos pos,
                                                T* __restrict__ out0, T* __restrict__ out1) {
  T v[P1];
#pragma unroll
  for (int k = 0; k < P1; ++k) v[k] = k < len ? u[pos(k)] : T(0);
#pragma unroll
  for (int k = 0; k < P1; ++k) {
    T se = 0, so = 0;
#pragma unroll
    for (int t = 0; k + t < P1; ++t) {
      if (t & 1) so = fma(shift_coef<T, 1>(t), v[k + t], so);
      else se = fma(shift_coef<T, 1>(t), v[k + t], se);
    }
    if (k < len) {
      const int q = pos(k);
      out0[q] = se - so;
      out1[q] = se + so;
    }
  }
}

__host__ __device__ inline int l2l_elems(int nj, int nfull) {
  return (7 * nfull + 8 * nj + 3) & ~3;  // Dt, 2 + 4 partial shifts, 8 children
}

template <typename T, int P>
__global__ void __launch_bounds__(32 * kWarps) k_l2l_w(PlanDev pd, const Geom* __restrict__ g,
                                                       int l, const double* __restrict__ lcp,
                                                       double* __restrict__ lcc) {
  constexpr int P1 = P + 1;
  constexpr int NROW = P1 * (P1 + 1) / 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nl = 1 << l;
  const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (b >= (int64_t)nl * nl * nl) return;
  const int c = min(pd.c, P1), nj = pd.nj, nfull = pd.nfull;
  extern __shared__ __align__(16) unsigned char smw[];
  T* D = reinterpret_cast<T*>(smw) + (size_t)warp * l2l_elems(nj, nfull);  // [nfull] Dt = M Lt
  T* X = D + nfull;                                                        // [2][nfull] (sx)
  T* Y = X + 2 * nfull;                                                    // [4][nfull] (sx + 2 sy)
  T* O = Y + 4 * nfull;                                                    // [8][nj] children
  for (int q = lane; q < nj; q += 32) D[q] = (T)lcp[b * nj + q];
  __syncwarp();
  decompress_warp<T>(pd, D, __dmul_rn(g->size, pow2_neg<double>(l)), lane);
  // x: rows of the full layout
  for (int r = lane; r < NROW; r += 32) {
    int ms, m1;
    pair_of<P1>(r, ms, m1);
    const int st = fpos<P1>(ms, m1, 0);
    shift_down_pair<T, P1>(D + st, P1 - ms - m1, [](int k) { return k; }, X + st, X + nfull + st);
  }
  __syncwarp();
  // y: columns (m_s, m_0) of the full layout, both x variants
  for (int sx = 0; sx < 2; ++sx)
    for (int r = lane; r < NROW; r += 32) {
      int ms, a;
      pair_of<P1>(r, ms, a);
      shift_down_pair<T, P1>(X + sx * nfull, P1 - ms - a,
                             [&](int k) { return fpos<P1>(ms, k, a); }, Y + sx * nfull,
                             Y + (sx + 2) * nfull);
    }
  __syncwarp();
  // slow axis: pillars (m_1, m_0) into the stored slabs of the 8 children
  // (child ci = v + 4 sz, v = sx + 2 sy), rescaled by 2^-|i|
  for (int v = 0; v < 4; ++v)
    for (int r = lane; r < NROW; r += 32) {
      int m1, a;
      pair_of<P1>(r, m1, a);
      const int len = P1 - m1 - a, cc = min(c, len);
      const T* yv = Y + v * nfull;
      T y[P1];
#pragma unroll
      for (int qs = 0; qs < P1; ++qs) y[qs] = qs < len ? yv[fpos<P1>(qs, m1, a)] : T(0);
#pragma unroll
      for (int is = 0; is < P1; ++is) {
        if (is < cc) {
          T se = 0, so = 0;
#pragma unroll
          for (int t = 0; is + t < P1; ++t) {
            if (t & 1) so = fma(shift_coef<T, 1>(t), y[is + t], so);
            else se = fma(shift_coef<T, 1>(t), y[is + t], se);
          }
          const T sc = pow2_neg<T>(a + m1 + is);
          const int q = fpos<P1>(is, m1, a);
          O[v * nj + q] = (se - so) * sc;
          O[(v + 4) * nj + q] = (se + so) * sc;
        }
      }
    }
  __syncwarp();
  const int bx = (int)(b & (nl - 1)), by = (int)((b >> l) & (nl - 1)), bz = (int)(b >> (2 * l));
  const int64_t nlc = 2 * (int64_t)nl;
  for (int ci = 0; ci < 8; ++ci) {
    const int64_t cb =
        ((2 * bz + (ci >> 2)) * nlc + (2 * by + ((ci >> 1) & 1))) * nlc + (2 * bx + (ci & 1));
    double* dst = lcc + cb * nj;
    const T* src = O + ci * nj;
    for (int q = lane; q < nj; q += 32) dst[q] += (double)src[q];
  }
}

// ---------------------------------------------------------------------------
// P2M, segments of monomials, two sources per instruction.
// ---------------------------------------------------------------------------
constexpr int kSeg = 4;

__host__ __device__ inline int p2m_floats(int p, int nfull) {
  const int ps = (p + 1) | 1;  // odd pitch (in float2) of the per-pair power tables
  return 3 * 16 * ps * 2 + ((nfull + 3) & ~3);
}

__device__ __forceinline__ f2_t lds2(const float2* p) {
  return *reinterpret_cast<const f2_t*>(p);
}

// the segment P2M of one box of side `side` with sources i0..i1: load(j)
// gives source j's (c - y)/s (x, y, z) and weight (w); the compressed
// box-scaled multipole goes to out
template <typename Load>
__device__ void p2m_seg_body(const PlanDev& pd, double side, int i0, int i1, Load load,
                             float* base, int lane, double* __restrict__ out) {
  const int p = pd.p, nfull = pd.nfull, nj = pd.nj, nseg = pd.p2m_nseg;
  const int ps = (p + 1) | 1;
  float2* TX = reinterpret_cast<float2*>(base);  // [16 source pairs][ps]: x^e
  float2* TY = TX + 16 * ps;                     // w y^e
  float2* TZ = TY + 16 * ps;                     // z^e
  float* alpha = base + 3 * 16 * ps * 2;
  if (i0 == i1) {
    for (int q = lane; q < nj; q += 32) out[q] = 0.0;
    return;
  }
  for (int q = lane; q < nfull; q += 32) alpha[q] = 0.f;
  for (int j0 = i0; j0 < i1; j0 += 32) {
    const int n = min(32, i1 - j0);
    __syncwarp();
    {  // lane j: powers of source j0 + j; past the end, weight 0
      const float4 r = lane < n ? load(j0 + lane) : make_float4(0.f, 0.f, 0.f, 0.f);
      const float ux = r.x, uy = r.y, uz = r.z;
      float vx = 1.f, vy = r.w, vz = 1.f;
      float* px = reinterpret_cast<float*>(TX + (lane >> 1) * ps) + (lane & 1);
      float* py = reinterpret_cast<float*>(TY + (lane >> 1) * ps) + (lane & 1);
      float* pz = reinterpret_cast<float*>(TZ + (lane >> 1) * ps) + (lane & 1);
      for (int e = 0; e <= p; ++e) {
        px[2 * e] = vx;
        py[2 * e] = vy;
        pz[2 * e] = vz;
        vx *= ux;
        vy *= uy;
        vz *= uz;
      }
    }
    __syncwarp();
    const int npair = (n + 1) >> 1;
    for (int s0 = lane; s0 < nseg; s0 += 64) {
      const int d0 = pd.p2m_seg[s0];
      const int d1 = s0 + 32 < nseg ? pd.p2m_seg[s0 + 32] : 0;  // len 0: nothing written
      const int a0 = d0 & 31, y0 = (d0 >> 5) & 31, z0 = (d0 >> 10) & 31;
      const int a1 = d1 & 31, y1 = (d1 >> 5) & 31, z1 = (d1 >> 10) & 31;
      f2_t acc0[kSeg], acc1[kSeg];
#pragma unroll
      for (int e = 0; e < kSeg; ++e) acc0[e] = acc1[e] = 0ull;
      for (int jp = 0; jp < npair; ++jp) {
        const float2* X = TX + jp * ps;
        const float2* Yt = TY + jp * ps;
        const float2* Z = TZ + jp * ps;
        const f2_t x = lds2(X + 1);
        f2_t v0 = f2mul(f2mul(lds2(X + a0), lds2(Yt + y0)), lds2(Z + z0));
        f2_t v1 = f2mul(f2mul(lds2(X + a1), lds2(Yt + y1)), lds2(Z + z1));
#pragma unroll
        for (int e = 0; e < kSeg; ++e) {
          acc0[e] = f2add(acc0[e], v0);
          acc1[e] = f2add(acc1[e], v1);
          if (e + 1 < kSeg) {
            v0 = f2mul(v0, x);
            v1 = f2mul(v1, x);
          }
        }
      }
      const int len0 = (d0 >> 15) & 7, pos0 = d0 >> 18;
      const int len1 = (d1 >> 15) & 7, pos1 = d1 >> 18;
#pragma unroll
      for (int e = 0; e < kSeg; ++e) {
        float lo, hi;
        if (e < len0) {
          f2unpack(acc0[e], lo, hi);
          alpha[pos0 + e] += lo + hi;
        }
        if (e < len1) {
          f2unpack(acc1[e], lo, hi);
          alpha[pos1 + e] += lo + hi;
        }
      }
    }
  }
  __syncwarp();
  for (int q = lane; q < nfull; q += 32) alpha[q] *= pd.inv_fact_f[q];
  __syncwarp();
  compress_warp<float>(pd, alpha, side, lane);
  for (int q = lane; q < nj; q += 32) out[q] = (double)alpha[q];
}

// uniform tree: the leaves' box-relative float copies (y - c)/s
__global__ void __launch_bounds__(32 * kWarps) k_p2m_seg(PlanDev pd, const Geom* __restrict__ g,
                                                         int64_t nleaf,
                                                         const int* __restrict__ start,
                                                         const float4* __restrict__ rel,
                                                         double* __restrict__ mp) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (b >= nleaf) return;
  extern __shared__ __align__(16) float smf[];
  p2m_seg_body(
      pd, g->s_leaf, start[b], start[b + 1],
      [&](int j) {
        const float4 r = rel[j];
        return make_float4(-r.x, -r.y, -r.z, r.w);
      },
      smf + (size_t)warp * p2m_floats(pd.p, pd.nfull), lane, mp + b * pd.nj);
}

// adaptive tree: every leaf of level >= 2, (c - y)/s from the FP64 sorted
// sources (one FP64 subtraction and product per coordinate)
__global__ void __launch_bounds__(32 * kWarps) k_ap2m_seg(PlanDev pd, const Geom* __restrict__ g,
                                                          ATree t, const double* __restrict__ x0,
                                                          const double* __restrict__ x1,
                                                          const double* __restrict__ x2,
                                                          const double* __restrict__ w,
                                                          double* __restrict__ mp) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = t.loff[2] + blockIdx.x * (blockDim.x >> 5) + warp;
  if (b >= t.loff[t.maxlev + 1] || !t.leaf[b] || t.s1[b] == t.s0[b]) return;
  int l, bc[3];
  abox(t, b, &l, bc);
  double c[3], s;
  abox_center(g, l, bc, c, &s);
  const double inv_s = 1.0 / s;
  extern __shared__ __align__(16) float smf[];
  p2m_seg_body(
      pd, s, t.s0[b], t.s1[b],
      [&](int j) {
        return make_float4((float)((c[0] - x0[j]) * inv_s), (float)((c[1] - x1[j]) * inv_s),
                           (float)((c[2] - x2[j]) * inv_s), (float)w[j]);
      },
      smf + (size_t)warp * p2m_floats(pd.p, pd.nfull), lane, mp + (size_t)b * pd.nj);
}

// ---------------------------------------------------------------------------
// L2P: nested Horner over the decompressed Lt_m / m! of the target's leaf.
// ---------------------------------------------------------------------------
constexpr int kL2pLeaves = 4;

template <int P, bool GRAD>
__device__ __forceinline__ float l2p_horner(const float* __restrict__ cb, float u0, float u1,
                                            float u2, float* gr) {
  constexpr int P1 = P + 1;
  float F = 0.f, F0 = 0.f, F1 = 0.f, F2 = 0.f;
#pragma unroll
  for (int ms = P; ms >= 0; --ms) {
    float S = 0.f, S0 = 0.f, S1 = 0.f;
#pragma unroll
    for (int m1 = P - ms; m1 >= 0; --m1) {
      const int len = P1 - ms - m1;
      const int bs = fpos<P1>(ms, m1, 0);
      float v = cb[bs + len - 1], dv = 0.f;
#pragma unroll
      for (int k = len - 2; k >= 0; --k) {
        if (GRAD) dv = fmaf(dv, u0, v);
        v = fmaf(v, u0, cb[bs + k]);
      }
      if (GRAD) {
        S1 = fmaf(S1, u1, S);
        S0 = fmaf(S0, u1, dv);
      }
      S = fmaf(S, u1, v);
    }
    if (GRAD) {
      F2 = fmaf(F2, u2, F);
      F0 = fmaf(F0, u2, S0);
      F1 = fmaf(F1, u2, S1);
    }
    F = fmaf(F, u2, S);
  }
  if (GRAD) {
    gr[0] = F0;
    gr[1] = F1;
    gr[2] = F2;
  }
  return F;
}

template <int P, bool GRAD>
__global__ void __launch_bounds__(32 * kWarps) k_l2p_f32(
    PlanDev pd, const Geom* __restrict__ g, int64_t nleaf, const double* __restrict__ lc,
    const int* __restrict__ tstart, const float4* __restrict__ txr, const int* __restrict__ tperm,
    double* __restrict__ phi, double* __restrict__ grad) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t b0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * kL2pLeaves;
  if (b0 >= nleaf) return;
  const int nb = (int)min((int64_t)kL2pLeaves, nleaf - b0);
  const int nj = pd.nj, nfull = pd.nfull;
  const int pitch = nfull | 1;  // odd: the leaves' tables start in different banks
  extern __shared__ __align__(16) float smf[];
  float* T = smf + (size_t)warp * kL2pLeaves * pitch;
  int bnd[kL2pLeaves];  // first target of each leaf (leaves past nb: the end)
#pragma unroll
  for (int k = 0; k < kL2pLeaves; ++k) bnd[k] = tstart[b0 + min(k, nb)];
  const int tend = tstart[b0 + nb];
  if (bnd[0] == tend) return;  // no targets in these leaves (warp-uniform)
  for (int k = 0; k < nb; ++k)
    for (int q = lane; q < nj; q += 32) T[k * pitch + q] = (float)lc[(b0 + k) * nj + q];
  __syncwarp();
  {  // decompression (eq. (decompression)) of the nb tables, slab by slab
    const int nt = pd.nterms > 0 ? pd.nterms : 1;
    float cf[FMM_MAX_TERMS];
    for (int t = 0; t < pd.nterms; ++t) cf[t] = scaled_coef_t<float>(pd, t, g->s_leaf);
    for (int ms = pd.c; ms <= pd.p; ++ms) {
      const int s0 = slab_begin(pd, ms), s1 = slab_begin(pd, ms + 1);
      for (int k = 0; k < nb; ++k) {
        float* Tk = T + k * pitch;
        for (int i = s0 + lane; i < s1; i += 32) {
          float v = 0.f;
          for (int t = 0; t < pd.nterms; ++t) v += cf[t] * Tk[pd.rec_src[i * nt + t]];
          Tk[i] = v;
        }
      }
      __syncwarp();
    }
    for (int k = 0; k < nb; ++k)
      for (int q = lane; q < nfull; q += 32) T[k * pitch + q] *= pd.inv_fact_f[q];
    __syncwarp();
  }
  const double inv_s = g->inv_s_leaf;
  for (int t = bnd[0] + lane; t - lane < tend; t += 32) {
    const bool valid = t < tend;
    int k = 0;
#pragma unroll
    for (int j = 1; j < kL2pLeaves; ++j) k += (j < nb && t >= bnd[j]) ? 1 : 0;
    const float4 q = valid ? txr[t] : make_float4(0.f, 0.f, 0.f, 0.f);
    float gr[3];
    const float f = l2p_horner<P, GRAD>(T + k * pitch, q.x, q.y, q.z, gr);
    if (valid) {
      const int orig = tperm[t];
      if (phi) phi[orig] += (double)f;
      if (GRAD && grad)
        for (int a = 0; a < 3; ++a) grad[(size_t)orig * 3 + a] += (double)gr[a] * inv_s;
    }
  }
}

// shared memory per block for nw warps, with the block shrunk to fit 96 KB
template <typename K>
int warps_for(K kernel, size_t per_warp, size_t* smem) {
  int nw = kWarps;
  while (nw > 1 && per_warp * nw > 96 * 1024) nw >>= 1;
  *smem = per_warp * nw;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
  return nw;
}

template <typename T, int P>
void m2m_go(const fmm_plan_s* P_, const Workspace& ws, int l, cudaStream_t st) {
  const PlanDev& pd = P_->pd;
  size_t smem;
  const int nw = warps_for(k_m2m_w<T, P>, sizeof(T) * m2m_elems(pd.nj, pd.nfull), &smem);
  const int64_t n = nbox_at(3, l);
  k_m2m_w<T, P><<<(unsigned)((n + nw - 1) / nw), 32 * nw, smem, st>>>(
      pd, ws.geom, l, ws.mp + ws.lev_off[l + 1] * pd.nj, ws.mp + ws.lev_off[l] * pd.nj);
}

template <typename T, int P>
void l2l_go(const fmm_plan_s* P_, const Workspace& ws, int l, cudaStream_t st) {
  const PlanDev& pd = P_->pd;
  size_t smem;
  const int nw = warps_for(k_l2l_w<T, P>, sizeof(T) * l2l_elems(pd.nj, pd.nfull), &smem);
  const int64_t n = nbox_at(3, l);
  k_l2l_w<T, P><<<(unsigned)((n + nw - 1) / nw), 32 * nw, smem, st>>>(
      pd, ws.geom, l, ws.lc + ws.lev_off[l] * pd.nj, ws.lc + ws.lev_off[l + 1] * pd.nj);
}

template <int P, bool GRAD>
void l2p_go(const fmm_plan_s* P_, const Workspace& ws, double* phi, double* grad,
            cudaStream_t st) {
  const PlanDev& pd = P_->pd;
  const int L = P_->desc.levels;
  const int64_t nleaf = nbox_at(3, L);
  size_t smem;
  const int nw = warps_for(k_l2p_f32<P, GRAD>,
                           sizeof(float) * kL2pLeaves * (size_t)(pd.nfull | 1), &smem);
  const int64_t nwarp = (nleaf + kL2pLeaves - 1) / kL2pLeaves;
  k_l2p_f32<P, GRAD><<<(unsigned)((nwarp + nw - 1) / nw), 32 * nw, smem, st>>>(
      pd, ws.geom, nleaf, ws.lc + ws.lev_off[L] * pd.nj, ws.tstart, ws.txr, ws.tperm, phi, grad);
}

#define PASSES_DISPATCH(PV, CALL) \
  switch (PV) {                   \
    case 4: CALL(4); break;       \
    case 6: CALL(6); break;       \
    case 8: CALL(8); break;       \
    case 10: CALL(10); break;     \
    case 12: CALL(12); break;     \
    case 16: CALL(16); break;     \
    default: return false;        \
  }

}  // namespace

bool passes_f32_order(int p) {
  return p == 4 || p == 6 || p == 8 || p == 10 || p == 12 || p == 16;
}

bool launch_p2m_f32(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st) {
  const PlanDev& pd = P->pd;
  if (pd.d != 3 || !ws.sxr || pd.p2m_nseg <= 0) return false;
  const int L = P->desc.levels;
  const int64_t nleaf = nbox_at(3, L);
  size_t smem;
  const int nw = warps_for(k_p2m_seg, sizeof(float) * p2m_floats(pd.p, pd.nfull), &smem);
  k_p2m_seg<<<(unsigned)((nleaf + nw - 1) / nw), 32 * nw, smem, st>>>(
      pd, ws.geom, nleaf, ws.sstart, ws.sxr, ws.mp + ws.lev_off[L] * pd.nj);
  return true;
}

bool launch_ap2m_f32(const fmm_plan_s* P, const Workspace& ws, const ATree& t, cudaStream_t st) {
  const PlanDev& pd = P->pd;
  if (pd.d != 3 || pd.p2m_nseg <= 0 || t.maxlev < 2) return false;
  const int n = t.loff[t.maxlev + 1] - t.loff[2];
  size_t smem;
  const int nw = warps_for(k_ap2m_seg, sizeof(float) * p2m_floats(pd.p, pd.nfull), &smem);
  k_ap2m_seg<<<(unsigned)((n + nw - 1) / nw), 32 * nw, smem, st>>>(pd, ws.geom, t, ws.sx[0],
                                                                    ws.sx[1], ws.sx[2], ws.sw,
                                                                    ws.mp);
  return true;
}

bool launch_m2m_warp(const fmm_plan_s* P, const Workspace& ws, int l, ShiftArith a,
                     cudaStream_t st) {
  if (P->pd.d != 3) return false;
  if (a == kShiftF64) {
#define GO(PP) m2m_go<double, PP>(P, ws, l, st)
    PASSES_DISPATCH(P->pd.p, GO)
#undef GO
  } else if (a == kShiftDW) {
#define GO(PP) m2m_go<dwf, PP>(P, ws, l, st)
    PASSES_DISPATCH(P->pd.p, GO)
#undef GO
  } else {
#define GO(PP) m2m_go<float, PP>(P, ws, l, st)
    PASSES_DISPATCH(P->pd.p, GO)
#undef GO
  }
  return true;
}

bool launch_l2l_warp(const fmm_plan_s* P, const Workspace& ws, int l, ShiftArith a,
                     cudaStream_t st) {
  if (P->pd.d != 3) return false;
  if (a == kShiftF64) {
#define GO(PP) l2l_go<double, PP>(P, ws, l, st)
    PASSES_DISPATCH(P->pd.p, GO)
#undef GO
  } else if (a == kShiftDW) {
#define GO(PP) l2l_go<dwf, PP>(P, ws, l, st)
    PASSES_DISPATCH(P->pd.p, GO)
#undef GO
  } else {
#define GO(PP) l2l_go<float, PP>(P, ws, l, st)
    PASSES_DISPATCH(P->pd.p, GO)
#undef GO
  }
  return true;
}

bool launch_l2p_f32(const fmm_plan_s* P, const Workspace& ws, double* phi, double* grad,
                    cudaStream_t st) {
  if (P->pd.d != 3 || !ws.txr) return false;
  if (grad) {
#define GO(PP) l2p_go<PP, true>(P, ws, phi, grad, st)
    PASSES_DISPATCH(P->pd.p, GO)
#undef GO
  } else {
#define GO(PP) l2p_go<PP, false>(P, ws, phi, grad, st)
    PASSES_DISPATCH(P->pd.p, GO)
#undef GO
  }
  return true;
}
