// M2L in its convolution form (Sec. 4.1, eq. (convolution_m2l)).
//
// For i, q in j the translation Lt_i = sum_q Ht[i + q] bt_q is a correlation
// of the multipole with the derivative table.  Reflecting the multipole
// (b'[-q] = bt_q) turns it into a d-dimensional convolution of sizes
// (M_a + 1), M = (p, p, c - 1), which a circular convolution of lengths
// n_a = 2 M_a + 1 reproduces without wrap-around for every i in j.  With
// E(x) = exp(2 pi i x) the transforms are
//     Bhat[k] = sum_{q in j} g^{|q|} bt_q E(+k.q/n)          (reflection folded in)
//     Hhat[k] = sum_{|m| <= 2p, m_s <= 2c-2} g^{-|m|} Ht[m] E(-k.m/n) / prod(n)
//     Lt_i    = g^{|i|} sum_k Hhat[k] Bhat[k] E(+k.i/n)
// where g is the scaling of Sec. 4.1.1.  Because every transformed array is
// real, only the Hermitian half k_0 = 0..p of the m_0 axis is kept.
//
// Work per evaluation:
//   k_fft_fwd     one block per box of levels 2..L: pruned separable DFT of
//                 its |j| coefficients (only the stored set is non-zero);
//   k_fft_htab    one block per (table level, offset): the same for the
//                 derivative tables;
//   k_fft_stencil per frequency, the interaction-list sum
//                 Ghat_t = sum_{h in V(t)} Hhat_h Bhat_{t-h} over the box grid;
//   k_fft_inv     one block per target box: pruned inverse DFT that produces
//                 only the i in j, scaled by g^{|i|}.
#include <algorithm>

#include "expansions.cuh"

namespace {

template <typename T>
struct Cplx;
template <>
struct Cplx<float> {
  using type = float2;
};
template <>
struct Cplx<double> {
  using type = double2;
};
template <typename T>
using C2 = typename Cplx<T>::type;

__device__ __forceinline__ float ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double ffma(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T>
__device__ __forceinline__ C2<T> cmk(T x, T y) {
  C2<T> r;
  r.x = x;
  r.y = y;
  return r;
}

// acc += a * b
template <typename T>
__device__ __forceinline__ void cmac(C2<T>& acc, const C2<T>& a, const C2<T>& b) {
  acc.x = ffma(a.x, b.x, acc.x);
  acc.x = ffma(-a.y, b.y, acc.x);
  acc.y = ffma(a.x, b.y, acc.y);
  acc.y = ffma(a.y, b.x, acc.y);
}

// acc += x * (e.x + i sg e.y)
template <typename T>
__device__ __forceinline__ void cmac_tw(C2<T>& acc, const C2<T>& x, const C2<T>& e, T sg) {
  const T ey = sg * e.y;
  acc.x = ffma(x.x, e.x, acc.x);
  acc.x = ffma(-x.y, ey, acc.x);
  acc.y = ffma(x.x, ey, acc.y);
  acc.y = ffma(x.y, e.x, acc.y);
}

constexpr int kThreads = 128;
constexpr int kTX = 8;  // target boxes along x per thread in the stencil

template <typename T>
__device__ void load_twiddles(const FftDev& f, C2<T>* tw1, C2<T>* tw3) {
  for (int i = threadIdx.x; i < f.n1; i += blockDim.x)
    tw1[i] = cmk<T>((T)f.tw1[2 * i], (T)f.tw1[2 * i + 1]);
  for (int i = threadIdx.x; i < f.n3; i += blockDim.x)
    tw3[i] = cmk<T>((T)f.tw3[2 * i], (T)f.tw3[2 * i + 1]);
}

// Pruned separable forward DFT of a real array a on the slab layout of order
// P with S slabs (row bases rb[ms*(P+1) + m1], d = 2: rb[ms]):
//     out[(k3*n2 + k2)*k1n + k] = sum_m a[m] E(sg (k m0/n1 + k2 m1/n2 + k3 ms/n3))
// for k < k1n = p + 1, k2 < n2, k3 < n3; entries kf..kfp-1 of out are zeroed.
// X holds S*(P+1)*k1n values; Y (S*n2*k1n values, d = 3 only) may alias a.
template <int D, typename T>
__device__ void dft_forward(const FftDev& f, const T* a, const int* rb, int P, int S, T sg,
                            const C2<T>* tw1, const C2<T>* tw3, C2<T>* X, C2<T>* Y,
                            C2<T>* __restrict__ out) {
  const int K1 = f.k1, n1 = f.n1, n2 = f.n2, n3 = f.n3;
  const int nr = D == 3 ? P + 1 : 1;  // rows per slab
  // axis m0 (real input)
  for (int w = threadIdx.x; w < S * nr * K1; w += blockDim.x) {
    const int k = w % K1, r = w / K1;
    const int m1 = D == 3 ? r % nr : 0, ms = D == 3 ? r / nr : r;
    const int len = P - ms - m1 + 1;
    T cx = 0, sx = 0;
    if (len > 0) {
      const T* row = a + (D == 3 ? rb[ms * (P + 1) + m1] : rb[ms]);
      int ph = 0;
      for (int m0 = 0; m0 < len; ++m0) {
        const C2<T> e = tw1[ph];
        cx = ffma(row[m0], e.x, cx);
        sx = ffma(row[m0], e.y, sx);
        ph += k;
        if (ph >= n1) ph -= n1;
      }
    }
    X[w] = cmk<T>(cx, sg * sx);
  }
  __syncthreads();
  // axis m1 (d = 3)
  const C2<T>* Ys = X;
  if (D == 3) {
    for (int w = threadIdx.x; w < S * n2 * K1; w += blockDim.x) {
      const int k = w % K1, k2 = (w / K1) % n2, ms = w / (K1 * n2);
      C2<T> acc = cmk<T>(0, 0);
      int ph = 0;
      for (int m1 = 0; m1 <= P - ms; ++m1) {
        cmac_tw<T>(acc, X[(ms * nr + m1) * K1 + k], tw1[ph], sg);
        ph += k2;
        if (ph >= n2) ph -= n2;
      }
      Y[w] = acc;
    }
    __syncthreads();
    Ys = Y;
  }
  // axis m_s, straight to global memory
  for (int w = threadIdx.x; w < f.kfp; w += blockDim.x) {
    C2<T> acc = cmk<T>(0, 0);
    if (w < f.kf) {
      const int k = w % K1, k2 = (w / K1) % n2, k3 = w / (K1 * n2);
      int ph = 0;
      for (int ms = 0; ms < S; ++ms) {
        cmac_tw<T>(acc, Ys[(ms * n2 + k2) * K1 + k], tw3[ph], sg);
        ph += k3;
        if (ph >= n3) ph -= n3;
      }
    }
    out[w] = acc;
  }
}

// number of stored slabs (m_s < c, at most p + 1)
__host__ __device__ inline int stored_slabs(const PlanDev& pd) {
  return pd.c < pd.p + 1 ? pd.c : pd.p + 1;
}

// ---------------------------------------------------------------------------
// Multipole spectra: one block per box of levels 2..L (global box index b).
// ---------------------------------------------------------------------------
template <int D, typename T>
__global__ void __launch_bounds__(kThreads) k_fft_fwd(PlanDev pd, FftDev f,
                                                      const double* __restrict__ mp,
                                                      C2<T>* __restrict__ bh) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int64_t b = blockIdx.x;
  const int S = stored_slabs(pd), P = pd.p;
  const int nr = D == 3 ? P + 1 : 1;
  C2<T>* tw1 = reinterpret_cast<C2<T>*>(smraw);
  C2<T>* tw3 = tw1 + f.n1;
  C2<T>* X = tw3 + f.n3;
  C2<T>* Y = X + S * nr * f.k1;  // also holds the input a
  T* a = reinterpret_cast<T*>(Y);
  load_twiddles<T>(f, tw1, tw3);
  for (int i = threadIdx.x; i < pd.nj; i += blockDim.x)
    a[i] = (T)(mp[b * pd.nj + i] * f.gpow[pd.mi[i].w]);
  __syncthreads();
  dft_forward<D, T>(f, a, pd.frow, P, S, (T)1, tw1, tw3, X, Y, bh + b * f.kfp);
}

// ---------------------------------------------------------------------------
// Offset-table spectra: block (offset o, table level tl); adjacent offsets
// (never in an interaction list) are skipped.  1/prod(n) is folded in.
// ---------------------------------------------------------------------------
template <int D, typename T>
__global__ void __launch_bounds__(kThreads) k_fft_htab(PlanDev pd, FftDev f,
                                                       const double* __restrict__ htab,
                                                       C2<T>* __restrict__ hh) {
  constexpr int NOFF = D == 3 ? 343 : 49;
  const int o = blockIdx.x, tl = blockIdx.y;
  {
    int t = o;
    bool adj = true;
    for (int k = 0; k < D; ++k) {
      const int dd = t % 7 - 3;
      t /= 7;
      if (dd < -1 || dd > 1) adj = false;
    }
    if (adj) return;
  }
  extern __shared__ __align__(16) unsigned char smraw[];
  const int P = 2 * pd.p, S = 2 * stored_slabs(pd) - 1;
  const int nr = D == 3 ? P + 1 : 1;
  C2<T>* tw1 = reinterpret_cast<C2<T>*>(smraw);
  C2<T>* tw3 = tw1 + f.n1;
  C2<T>* X = tw3 + f.n3;
  C2<T>* Y = X + S * nr * f.k1;
  T* a = reinterpret_cast<T*>(Y);
  load_twiddles<T>(f, tw1, tw3);
  const double inv_n = 1.0 / ((double)f.n1 * f.n2 * f.n3);
  const double* src = htab + ((size_t)tl * NOFF + o) * pd.nh;
  const double* gneg = f.gpow + (2 * pd.p + 1);
  for (int r = threadIdx.x; r < S * nr; r += blockDim.x) {
    const int m1 = D == 3 ? r % nr : 0, ms = D == 3 ? r / nr : r;
    const int len = P - ms - m1 + 1;
    if (len <= 0) continue;
    const int base = D == 3 ? pd.hrow[ms * (P + 1) + m1] : pd.hrow[ms];
    for (int m0 = 0; m0 < len; ++m0)
      a[base + m0] = (T)(src[base + m0] * gneg[ms + m1 + m0] * inv_n);
  }
  __syncthreads();
  dft_forward<D, T>(f, a, pd.hrow, P, S, (T)-1, tw1, tw3, X, Y,
                    hh + ((size_t)tl * NOFF + o) * f.kfp);
}

// ---------------------------------------------------------------------------
// Interaction-list sum per frequency.  A warp owns 32 consecutive
// frequencies of a strip of kTX target boxes along x at fixed (y, z); it
// walks the rows (hy, hz) of offsets allowed by the parities of (ty, tz) --
// h_a in [-3, 2] for an even target coordinate, [-2, 3] for an odd one
// (children of the parent's neighbours) -- loads the kTX + 6 source spectra
// of the row once and reuses each for up to 6 targets.  In rows with
// |hy|, |hz| <= 1 only |hx| >= 2 is taken (not adjacent to the target).
// ---------------------------------------------------------------------------
struct StLevel {
  int n;            // boxes per axis
  int nsx;          // strips along x
  int first_block;  // first blockIdx.x of the level
  int tl;           // table level
  int64_t off;      // first global box of the level
  double scale;     // table scale of the level (homogeneous kernels)
};
struct StParams {
  int nlev;
  StLevel lev[FMM_MAX_LEVELS];
};

template <typename T, bool NEAR>
__device__ __forceinline__ void row_mac(C2<T> (&acc)[kTX], const C2<T> (&H)[7],
                                        const C2<T> (&B)[kTX + 6]) {
#pragma unroll
  for (int j = 0; j < kTX; ++j) {
#pragma unroll
    for (int u = 0; u < 7; ++u) {
      const int hx = u - 3;
      const bool par = (j & 1) ? (hx >= -2) : (hx <= 2);
      const bool far = hx <= -2 || hx >= 2;
      if (par && (!NEAR || far)) cmac<T>(acc[j], H[u], B[j - u + 6]);
    }
  }
}

template <int D, typename T>
__global__ void __launch_bounds__(kThreads) k_fft_stencil(FftDev f, StParams prm,
                                                          const C2<T>* __restrict__ bh,
                                                          const C2<T>* __restrict__ hh,
                                                          C2<T>* __restrict__ gh) {
  constexpr int NOFF = D == 3 ? 343 : 49;
  int li = 0;
  while (li + 1 < prm.nlev && (int)blockIdx.x >= prm.lev[li + 1].first_block) ++li;
  const int n = prm.lev[li].n, nsx = prm.lev[li].nsx, tl = prm.lev[li].tl;
  const int64_t off = prm.lev[li].off;
  const T scale = (T)prm.lev[li].scale;
  const int strip = blockIdx.x - prm.lev[li].first_block;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kb = (blockIdx.y * (kThreads / 32) + warp) * 32;
  if (kb >= f.kfp) return;
  const int kfp = f.kfp;
  const int k = kb + lane;
  const int sx0 = (strip % nsx) * kTX;
  const int rest = strip / nsx;
  const int ty = D == 3 ? rest % n : rest;
  const int tz = D == 3 ? rest / n : 0;
  const C2<T>* hb = hh + (size_t)tl * NOFF * kfp + k;
  const C2<T>* bb = bh + (size_t)off * kfp + k;
  C2<T> acc[kTX];
#pragma unroll
  for (int j = 0; j < kTX; ++j) acc[j] = cmk<T>(0, 0);
  const int py = ty & 1, pz = tz & 1;
  const int hz0 = D == 3 ? -3 + pz : 0, hz1 = D == 3 ? 2 + pz : 0;
  for (int hz = hz0; hz <= hz1; ++hz) {
    const int sz = tz - hz;
    if (D == 3 && (sz < 0 || sz >= n)) continue;
    for (int hy = -3 + py; hy <= 2 + py; ++hy) {
      const int sy = ty - hy;
      if (sy < 0 || sy >= n) continue;
      const bool near = hy >= -1 && hy <= 1 && hz >= -1 && hz <= 1;
      const int ob = D == 3 ? ((hz + 3) * 7 + (hy + 3)) * 7 : (hy + 3) * 7;
      const int64_t rowb = ((int64_t)(D == 3 ? sz : 0) * n + sy) * n;
      C2<T> B[kTX + 6], H[7];
#pragma unroll
      for (int j = 0; j < kTX + 6; ++j) {
        const int sx = sx0 - 3 + j;
        B[j] = (sx >= 0 && sx < n) ? bb[(rowb + sx) * kfp] : cmk<T>(0, 0);
      }
      if (near) {
#pragma unroll
        for (int u = 0; u < 7; ++u)
          H[u] = (u <= 1 || u >= 5) ? hb[(size_t)(ob + u) * kfp] : cmk<T>(0, 0);
        row_mac<T, true>(acc, H, B);
      } else {
#pragma unroll
        for (int u = 0; u < 7; ++u) H[u] = hb[(size_t)(ob + u) * kfp];
        row_mac<T, false>(acc, H, B);
      }
    }
  }
  const int64_t tb = off + ((int64_t)(D == 3 ? tz : 0) * n + ty) * n;
#pragma unroll
  for (int j = 0; j < kTX; ++j) {
    const int tx = sx0 + j;
    if (tx < n) gh[(tb + tx) * kfp + k] = cmk<T>(acc[j].x * scale, acc[j].y * scale);
  }
}

// ---------------------------------------------------------------------------
// Local coefficients from the summed spectra: one block per target box.
// ---------------------------------------------------------------------------
template <int D, typename T>
__global__ void __launch_bounds__(kThreads) k_fft_inv(PlanDev pd, FftDev f,
                                                      const C2<T>* __restrict__ gh,
                                                      double* __restrict__ lc) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int64_t b = blockIdx.x;
  const int S = stored_slabs(pd), P = pd.p;
  const int K1 = f.k1, n1 = f.n1, n2 = f.n2, n3 = f.n3;
  const int nr = D == 3 ? P + 1 : 1;
  C2<T>* tw1 = reinterpret_cast<C2<T>*>(smraw);
  C2<T>* tw3 = tw1 + n1;
  C2<T>* Z = tw3 + n3;          // S x n2 x K1
  C2<T>* G = Z + S * n2 * K1;   // kf, later W (S x nr x K1)
  load_twiddles<T>(f, tw1, tw3);
  for (int w = threadIdx.x; w < f.kf; w += blockDim.x) G[w] = gh[b * f.kfp + w];
  __syncthreads();
  // axis m_s: Z[is][k2][k] = sum_k3 G[k3][k2][k] E(+k3 is/n3)
  for (int w = threadIdx.x; w < S * n2 * K1; w += blockDim.x) {
    const int k = w % K1, k2 = (w / K1) % n2, is = w / (K1 * n2);
    C2<T> acc = cmk<T>(0, 0);
    int ph = 0;
    for (int k3 = 0; k3 < n3; ++k3) {
      cmac_tw<T>(acc, G[(k3 * n2 + k2) * K1 + k], tw3[ph], (T)1);
      ph += is;
      if (ph >= n3) ph -= n3;
    }
    Z[w] = acc;
  }
  __syncthreads();
  // axis m1 (d = 3): W[is][i1][k] = sum_k2 Z[is][k2][k] E(+k2 i1/n2)
  const C2<T>* W = Z;
  if (D == 3) {
    C2<T>* Wd = G;
    for (int w = threadIdx.x; w < S * nr * K1; w += blockDim.x) {
      const int k = w % K1, i1 = (w / K1) % nr, is = w / (K1 * nr);
      C2<T> acc = cmk<T>(0, 0);
      if (i1 <= P - is) {
        int ph = 0;
        for (int k2 = 0; k2 < n2; ++k2) {
          cmac_tw<T>(acc, Z[(is * n2 + k2) * K1 + k], tw1[ph], (T)1);
          ph += i1;
          if (ph >= n2) ph -= n2;
        }
      }
      Wd[w] = acc;
    }
    __syncthreads();
    W = Wd;
  }
  // axis m0 (Hermitian half: weight 1 at k = 0, 2 elsewhere; n1 is odd)
  for (int i = threadIdx.x; i < pd.nj; i += blockDim.x) {
    const char4 m = pd.mi[i];
    const int i0 = m.x, i1 = D == 3 ? m.y : 0, is = D == 3 ? m.z : m.y;
    const C2<T>* row = W + (is * nr + i1) * K1;
    T v = row[0].x, v2 = 0;
    int ph = i0;
    for (int k = 1; k < K1; ++k) {
      const C2<T> e = tw1[ph];
      v2 = ffma(row[k].x, e.x, v2);
      v2 = ffma(-row[k].y, e.y, v2);
      ph += i0;
      if (ph >= n1) ph -= n1;
    }
    v = ffma((T)2, v2, v);
    lc[b * pd.nj + i] = (double)v * f.gpow[m.w];
  }
}

template <typename K>
void set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int D, typename T>
cudaError_t run_fft(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st, int* nl) {
  const PlanDev& pd = P->pd;
  const FftDev& f = P->fft;
  const int L = P->desc.levels;
  const int S = stored_slabs(pd), Sh = 2 * S - 1;
  const int nr = D == 3 ? pd.p + 1 : 1, nrh = D == 3 ? 2 * pd.p + 1 : 1;
  constexpr int NOFF = D == 3 ? 343 : 49;
  const size_t cs = sizeof(C2<T>);
  const int64_t nbox = ws.lev_off[L + 1];  // boxes of levels 2..L
  C2<T>* bh = static_cast<C2<T>*>(ws.fft_b);
  C2<T>* gh = static_cast<C2<T>*>(ws.fft_g);
  C2<T>* hh = static_cast<C2<T>*>(ws.fft_h);
  const bool shared = m2l_shared_tables(P);
  const int ntl = shared ? 1 : L - 1;

  // multipole spectra
  {
    const size_t yb = std::max(cs * S * f.n2 * f.k1, sizeof(T) * pd.nj);
    const size_t smem = cs * (f.n1 + f.n3) + cs * S * nr * f.k1 + yb;
    set_smem(k_fft_fwd<D, T>, smem);
    k_fft_fwd<D, T><<<(unsigned)nbox, kThreads, smem, st>>>(pd, f, ws.mp, bh);
    ++*nl;
  }
  // offset-table spectra
  {
    const size_t yb = std::max(cs * Sh * f.n2 * f.k1, sizeof(T) * pd.nh);
    const size_t smem = cs * (f.n1 + f.n3) + cs * Sh * nrh * f.k1 + yb;
    set_smem(k_fft_htab<D, T>, smem);
    k_fft_htab<D, T><<<dim3(NOFF, ntl), kThreads, smem, st>>>(pd, f, ws.htab, hh);
    ++*nl;
  }
  // interaction-list sums, all levels in one launch
  {
    StParams prm{};
    int nb = 0;
    for (int l = 2; l <= L; ++l) {
      StLevel& v = prm.lev[prm.nlev++];
      v.n = 1 << l;
      v.nsx = (v.n + kTX - 1) / kTX;
      v.first_block = nb;
      v.tl = shared ? 0 : l - 2;
      v.off = ws.lev_off[l];
      v.scale = 1.0;
      if (shared)  // Ht_l = Ht_2 * 2^{(l-2)}: 3D Laplace (degree -1); 2^{-(l-2)}: biharmonic
        v.scale = pd.kernel == FMM_KERNEL_LAPLACE ? std::ldexp(1.0, l - 2) : std::ldexp(1.0, 2 - l);
      nb += v.nsx * (D == 3 ? v.n * v.n : v.n);
    }
    const int kgroups = (f.kfp + kThreads - 1) / kThreads;
    mark_contraction(P, 0, st);
    k_fft_stencil<D, T><<<dim3(nb, kgroups), kThreads, 0, st>>>(f, prm, bh, hh, gh);
    mark_contraction(P, 1, st);
    ++*nl;
  }
  // local coefficients
  {
    const size_t gb = cs * std::max(f.kf, S * nr * f.k1);
    const size_t smem = cs * (f.n1 + f.n3) + cs * S * f.n2 * f.k1 + gb;
    set_smem(k_fft_inv<D, T>, smem);
    k_fft_inv<D, T><<<(unsigned)nbox, kThreads, smem, st>>>(pd, f, gh, ws.lc);
    ++*nl;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_m2l_fft(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st, int* nl) {
  const bool f64 = P->desc.precision == FMM_PREC_FP64;
  if (P->pd.d == 3) return f64 ? run_fft<3, double>(P, ws, st, nl) : run_fft<3, float>(P, ws, st, nl);
  return f64 ? run_fft<2, double>(P, ws, st, nl) : run_fft<2, float>(P, ws, st, nl);
}
