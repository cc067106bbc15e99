// M2L on the CUDA cores (Sec. 4.1, eq. (m2l_toeplitz), un-normalised):
//   Lt_t[i] += sum_{q in j} Ht_{l, t-s}[i + q] bt_s[q],   i in j,
// over the interaction list of every target box t: the children of the
// parent's neighbours (parent included) that are not adjacent to t.  The
// Hankel table Ht of the offset is staged in shared memory once per source,
// and each row (q_s, q_1) of the stored set is a contiguous run in both the
// table and the source coefficients, so the inner loop streams two arrays.
// One block per target box; used for the FP64 and FP32 configurations.
#include <algorithm>

#include "adaptive.cuh"
#include "expansions.cuh"

namespace {

constexpr int kThreads = 128;
constexpr int kMaxI = 8;  // stored terms per thread: 8 * 128 >= |j| for p <= 20

template <typename K>
void set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Accumulates one source box: stage its table row Ht (nh) and multipole
// bt (nj) in shared memory, then acc[k] += sum_q Ht[i_k + q] bt[q].
template <int D, typename T>
__device__ __forceinline__ void m2l_one_source(const PlanDev& pd, const double* __restrict__ hsrc,
                                               const double* __restrict__ bsrc, T* H, T* bs,
                                               T (&acc)[kMaxI], const int (&ii0)[kMaxI],
                                               const int (&ii1)[kMaxI], const int (&iis)[kMaxI]) {
  const int p = pd.p, c = pd.c, nj = pd.nj, nh = pd.nh, P2 = 2 * p;
  __syncthreads();
  for (int i = threadIdx.x; i < nh; i += blockDim.x) H[i] = (T)hsrc[i];
  for (int i = threadIdx.x; i < nj; i += blockDim.x) bs[i] = (T)bsrc[i];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kMaxI; ++k) {
    if (threadIdx.x + k * blockDim.x >= nj) continue;
    T sum = 0;
    for (int qs = 0; qs < c; ++qs) {
      if (D == 3) {
        for (int q1 = 0; q1 <= p - qs; ++q1) {
          const T* hrow = H + pd.hrow[(iis[k] + qs) * (P2 + 1) + ii1[k] + q1] + ii0[k];
          const T* brow = bs + pd.frow[qs * (p + 1) + q1];
          const int len = p - qs - q1 + 1;
          for (int q0 = 0; q0 < len; ++q0) sum += hrow[q0] * brow[q0];
        }
      } else {
        const T* hrow = H + pd.hrow[iis[k] + qs] + ii0[k];
        const T* brow = bs + pd.frow[qs];
        const int len = p - qs + 1;
        for (int q0 = 0; q0 < len; ++q0) sum += hrow[q0] * brow[q0];
      }
    }
    acc[k] += sum;
  }
}

template <int D, typename T>
__device__ __forceinline__ void m2l_init(const PlanDev& pd, T (&acc)[kMaxI], int (&ii0)[kMaxI],
                                         int (&ii1)[kMaxI], int (&iis)[kMaxI]) {
#pragma unroll
  for (int k = 0; k < kMaxI; ++k) {
    acc[k] = 0;
    const int i = threadIdx.x + k * blockDim.x;
    const char4 m = i < pd.nj ? pd.mi[i] : make_char4(0, 0, 0, 0);
    ii0[k] = m.x;
    ii1[k] = D == 3 ? m.y : 0;
    iis[k] = D == 3 ? m.z : m.y;
  }
}

template <int D, typename T>
__global__ void __launch_bounds__(kThreads) k_m2l_simt(PlanDev pd, int l,
                                                       const double* __restrict__ mp,
                                                       double* __restrict__ lc,
                                                       const double* __restrict__ htab) {
  const int b = blockIdx.x;
  const int nj = pd.nj, nh = pd.nh;
  const int nl = 1 << l;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* H = reinterpret_cast<T*>(smraw);
  T* bs = H + nh;
  int bc[3], pc[3];
  {
    int64_t t = b;
    for (int k = 0; k < D; ++k) {
      bc[k] = (int)(t % nl);
      t /= nl;
      pc[k] = bc[k] >> 1;
    }
  }
  T acc[kMaxI];
  int ii0[kMaxI], ii1[kMaxI], iis[kMaxI];
  m2l_init<D, T>(pd, acc, ii0, ii1, iis);
  int nn = 1;
  for (int k = 0; k < D; ++k) nn *= 6;
  for (int a = 0; a < nn; ++a) {
    int sc[3], tt = a, o = 0, mul = 1;
    bool ok = true, adj = true;
    for (int k = 0; k < D; ++k) {
      sc[k] = 2 * (pc[k] - 1) + tt % 6;
      tt /= 6;
      if (sc[k] < 0 || sc[k] >= nl) ok = false;
      const int dd = bc[k] - sc[k];
      if (dd > 1 || dd < -1) adj = false;
      o += (dd + 3) * mul;
      mul *= 7;
    }
    if (!ok || adj) continue;
    int64_t sb = 0;
    for (int k = D - 1; k >= 0; --k) sb = sb * nl + sc[k];
    m2l_one_source<D, T>(pd, htab + (size_t)o * nh, mp + (size_t)sb * nj, H, bs, acc, ii0, ii1,
                         iis);
  }
#pragma unroll
  for (int k = 0; k < kMaxI; ++k) {
    const int i = threadIdx.x + k * blockDim.x;
    if (i < nj) lc[(size_t)b * nj + i] += (double)acc[k];
  }
}

// Adaptive tree: one block per box of level >= 2 holding targets.  V(B) =
// children of the boxes adjacent to P(B) that are not adjacent to B, found by
// looking up the 27 neighbours of the parent; their offsets lie in [-3,3]^3.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_am2l(PlanDev pd, ATree t,
                                                   const double* __restrict__ mp,
                                                   double* __restrict__ lc,
                                                   const double* __restrict__ htab,
                                                   unsigned long long* __restrict__ count,
                                                   unsigned skip_mask) {
  const int b = t.loff[2] + blockIdx.x;
  if (b >= t.loff[t.maxlev + 1] || t.t1[b] == t.t0[b]) return;
  if ((skip_mask >> t.lev[b]) & 1u) return;  // done on the tensor cores
  const int nj = pd.nj, nh = pd.nh;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* H = reinterpret_cast<T*>(smraw);
  T* bs = H + nh;
  int l, bc[3];
  abox(t, b, &l, bc);
  const int pc[3] = {bc[0] >> 1, bc[1] >> 1, bc[2] >> 1};
  const double* ht = htab + (size_t)(l - 2) * 343 * nh;
  T acc[kMaxI];
  int ii0[kMaxI], ii1[kMaxI], iis[kMaxI];
  m2l_init<3, T>(pd, acc, ii0, ii1, iis);
  unsigned long long nv = 0;
  for (int nb = 0; nb < 27; ++nb) {
    const int nc[3] = {pc[0] + nb % 3 - 1, pc[1] + (nb / 3) % 3 - 1, pc[2] + nb / 9 - 1};
    const int Pn = alookup(t, l - 1, nc);
    if (Pn < 0 || t.leaf[Pn]) continue;
    for (int ci = 0; ci < 8; ++ci) {
      const int C = t.child[8 * Pn + ci];
      if (C < 0) continue;
      const int cc[3] = {2 * nc[0] + (ci & 1), 2 * nc[1] + ((ci >> 1) & 1),
                         2 * nc[2] + ((ci >> 2) & 1)};
      const int d0 = bc[0] - cc[0], d1 = bc[1] - cc[1], d2 = bc[2] - cc[2];
      if (d0 >= -1 && d0 <= 1 && d1 >= -1 && d1 <= 1 && d2 >= -1 && d2 <= 1) continue;
      const int o = (d0 + 3) + 7 * (d1 + 3) + 49 * (d2 + 3);
      m2l_one_source<3, T>(pd, ht + (size_t)o * nh, mp + (size_t)C * nj, H, bs, acc, ii0, ii1,
                           iis);
      ++nv;
    }
  }
  if (threadIdx.x == 0 && nv) atomicAdd(count, nv);
#pragma unroll
  for (int k = 0; k < kMaxI; ++k) {
    const int i = threadIdx.x + k * blockDim.x;
    if (i < nj) lc[(size_t)b * nj + i] += (double)acc[k];
  }
}

// The interaction-list sizes of the levels in `mask` (translated on the
// tensor cores, which run over whole windows and count nothing): one warp per
// box holding targets, lane n < 27 takes the n-th neighbour of the parent and
// counts its children that are not adjacent to the box.
constexpr int kCountWarps = 8;
__global__ void __launch_bounds__(32 * kCountWarps) k_am2l_count(ATree t, unsigned mask,
                                                                unsigned long long* count) {
  __shared__ unsigned long long blk;
  if (threadIdx.x == 0) blk = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int b = t.loff[2] + (int)(blockIdx.x * kCountWarps + (threadIdx.x >> 5));
  const bool live = b < t.loff[t.maxlev + 1] && t.t1[b] > t.t0[b] && ((mask >> t.lev[b]) & 1u);
  unsigned nv = 0;
  if (live && lane < 27) {
    int l, bc[3];
    abox(t, b, &l, bc);
    const int nc[3] = {(bc[0] >> 1) + lane % 3 - 1, (bc[1] >> 1) + (lane / 3) % 3 - 1,
                       (bc[2] >> 1) + lane / 9 - 1};
    const int Pn = alookup(t, l - 1, nc);
    if (Pn >= 0 && !t.leaf[Pn])
      for (int ci = 0; ci < 8; ++ci) {
        if (t.child[8 * Pn + ci] < 0) continue;
        const int d0 = bc[0] - (2 * nc[0] + (ci & 1)), d1 = bc[1] - (2 * nc[1] + ((ci >> 1) & 1)),
                  d2 = bc[2] - (2 * nc[2] + ((ci >> 2) & 1));
        nv += !(d0 >= -1 && d0 <= 1 && d1 >= -1 && d1 <= 1 && d2 >= -1 && d2 <= 1);
      }
  }
  nv = __reduce_add_sync(0xffffffffu, nv);
  if (lane == 0 && nv) atomicAdd(&blk, (unsigned long long)nv);
  __syncthreads();
  if (threadIdx.x == 0 && blk) atomicAdd(count, blk);
}

}  // namespace

cudaError_t launch_m2l_simt_levels(const fmm_plan_s* P, const Workspace& ws, int l0, int l1,
                                   cudaStream_t st, int* nl) {
  const PlanDev& pd = P->pd;
  const int d = pd.d;
  const bool f64 = P->desc.precision == FMM_PREC_FP64;
  const size_t tsz = f64 ? 8 : 4;
  const size_t smem = tsz * (pd.nh + pd.nj);
  const int noff = d == 3 ? 343 : 49;
  mark_contraction(P, 0, st);
  for (int l = l0; l <= l1; ++l) {
    const double* mpl = ws.mp + ws.lev_off[l] * pd.nj;
    double* lcl = ws.lc + ws.lev_off[l] * pd.nj;
    const double* ht = ws.htab + (size_t)(l - 2) * noff * pd.nh;
    const unsigned nb = (unsigned)nbox_at(d, l);
#define M2L_LAUNCH(DD, TT)                                                         \
  do {                                                                             \
    set_smem(k_m2l_simt<DD, TT>, smem);                                            \
    k_m2l_simt<DD, TT><<<nb, kThreads, smem, st>>>(pd, l, mpl, lcl, ht);           \
  } while (0)
    if (d == 3) {
      if (f64) M2L_LAUNCH(3, double); else M2L_LAUNCH(3, float);
    } else {
      if (f64) M2L_LAUNCH(2, double); else M2L_LAUNCH(2, float);
    }
#undef M2L_LAUNCH
    ++*nl;
  }
  mark_contraction(P, 1, st);
  return cudaGetLastError();
}

// M2L dispatcher: zero the local expansions of levels 2..L, then run the
// configured contraction path.
cudaError_t launch_m2l_tc(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st, int* nl,
                          bool tables_ready);
cudaError_t launch_m2l_tc_tables(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st,
                                 int* nl);

static bool uses_tc_tables(const fmm_plan_s* P) {
  const int prec = P->desc.precision;
  return P->desc.m2l != FMM_M2L_FFT && prec != FMM_PREC_FP64 && prec != FMM_PREC_FP32 &&
         P->pd.d == 3 && P->desc.levels > 0;
}

cudaError_t launch_m2l_tables(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st, int* nl) {
  return uses_tc_tables(P) ? launch_m2l_tc_tables(P, ws, st, nl) : cudaGetLastError();
}

cudaError_t launch_m2l(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st, int* nl,
                       bool tables_ready) {
  const int L = P->desc.levels;
  const int prec = P->desc.precision;
  const bool tc = P->desc.m2l != FMM_M2L_FFT && prec != FMM_PREC_FP64 && prec != FMM_PREC_FP32;
  // the tensor-core contraction stores every coefficient of levels 2..L once
  // (it zeroes the 2D fallback's expansions itself); the other forms add
  if (!tc) cudaMemsetAsync(ws.lc, 0, sizeof(double) * (size_t)ws.lev_off[L + 1] * P->pd.nj, st);
  if (P->desc.m2l == FMM_M2L_FFT) return launch_m2l_fft(P, ws, st, nl);
  if (!tc) return launch_m2l_simt_levels(P, ws, 2, L, st, nl);
  return launch_m2l_tc(P, ws, st, nl, tables_ready && uses_tc_tables(P));
}

cudaError_t launch_adaptive_m2l(const fmm_plan_s* P, const Workspace& ws, const ATree& t,
                                cudaStream_t st, int* nl) {
  const PlanDev& pd = P->pd;
  if (t.maxlev < 2) return cudaGetLastError();
  const unsigned nb = (unsigned)(t.loff[t.maxlev + 1] - t.loff[2]);
  const int prec = P->desc.precision;
  unsigned done = 0;
  mark_contraction(P, 0, st);
  if (prec_tensor(prec)) {
    const cudaError_t e = launch_adaptive_m2l_tc(P, ws, t, st, nl, &done);
    if (e != cudaSuccess) return e;
  }
  unsigned all = 0;
  for (int l = 2; l <= t.maxlev; ++l) all |= 1u << l;
  if (done) {  // interaction-list counts of the tensor-core levels
    k_am2l_count<<<(nb + kCountWarps - 1) / kCountWarps, 32 * kCountWarps, 0, st>>>(
        t, done, &ws.geom->m2l_count);
    ++*nl;
  }
  if ((done & all) != all) {
    if (prec == FMM_PREC_FP64) {
      const size_t smem = sizeof(double) * (pd.nh + pd.nj);
      set_smem(k_am2l<double>, smem);
      k_am2l<double><<<nb, kThreads, smem, st>>>(pd, t, ws.mp, ws.lc, ws.htab,
                                                 &ws.geom->m2l_count, done);
    } else {
      const size_t smem = sizeof(float) * (pd.nh + pd.nj);
      set_smem(k_am2l<float>, smem);
      k_am2l<float><<<nb, kThreads, smem, st>>>(pd, t, ws.mp, ws.lc, ws.htab,
                                                &ws.geom->m2l_count, done);
    }
    ++*nl;
  }
  mark_contraction(P, 1, st);
  return cudaGetLastError();
}
