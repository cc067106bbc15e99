// Tensor-core M2L (tcgen05, kind::tf32 / kind::f16) -- eq. (m2l_toeplitz) grouped by
// translation offset into dense contractions on the fifth-generation tensor
// cores, with the accumulator in TMEM.
//
// For a level with half-grid size H = 2^(l-1), write every box as 2T + pi
// (T its parent's coordinate, pi in {0,1}^3 its position in the parent).
// A target of class pi receives, from source child sigma of the parent
// T + delta (delta in {-1,0,1}^3), the translation with offset
// h = pi - sigma - 2 delta, whenever h is not adjacent (max |h_k| >= 2).
// For a fixed (pi, sigma, delta) the sources of a tile of targets T are the
// same tile of parents shifted by delta, so with the multipoles stored
// parity-split, Bpar[sigma][Tz][Ty][Tx][q], one 5-D TMA box (zero-filled
// outside the domain) is the B operand, and the dense offset matrix
//   A_h[i][q] = Ht_h[i + q]   (i, q in j)
// is the A operand.  One CTA owns one (tile of up to 256 target parents,
// pi, 128-row block of i), accumulates D[i][T] = sum_{sigma,delta,q}
// A_h[i][q] Bpar[...][q] per offset in TMEM, sums the offsets in registers and
// adds the result into the FP64 local expansions.
//
// Precision: TF32 (one pass), or TF32x3 / BF16x3 (a = a_hi + a_lo split,
// three passes a_hi b_hi + a_hi b_lo + a_lo b_hi), FP32 accumulation.
//
// Tile width.  An MMA of N = 256 columns reads its A slice once for twice the
// work of N = 128: the operand traffic out of shared memory drops from 128 to
// 96 bytes per clock at the full tensor rate, and each MMA runs twice as long,
// which leaves room for the issuing thread's barrier waits and commits between
// MMAs.  Measured on this kernel's issue pattern (three passes, one wait and
// one commit per stage), N = 128 kept the tensor pipe 85% busy and N = 256
// 99%.
#include <algorithm>
#include <cstring>

#include <cuda_bf16.h>

#include "adaptive.cuh"
#include "expansions.cuh"
#include "tc_ptx.cuh"

cudaError_t launch_m2l_simt_levels(const fmm_plan_s* P, const Workspace& ws, int l0, int l1,
                                   cudaStream_t st, int* nl);

namespace {

constexpr int kBM = 128;    // rows of A / TMEM lanes
constexpr int kMaxN = 256;  // target parents per CTA = MMA N

// Operand formats: tf32 (fp32 storage, 32 per 128-byte row, kind::tf32) and
// bf16 (64 per row, kind::f16).  Both split a value into hi + lo.
// The split works on the float rounding of the value (one conversion from
// FP64): lo = f - hi is exact in float, and keeps the bits the tf32/bf16
// format drops from hi.
struct FmtTF32 {
  using T = float;
  static constexpr int kRow = 32;
  static constexpr int kIdesc = 2;
  static constexpr bool kF16 = false;
  static __device__ __forceinline__ void split(float f, T& hi, T& lo) {
    const float h = tc::tf32_rna(f);
    hi = h;
    lo = tc::tf32_rna(f - h);
  }
};
struct FmtBF16 {
  using T = __nv_bfloat16;
  static constexpr int kRow = 64;
  static constexpr int kIdesc = 1;
  static constexpr bool kF16 = true;
  static __device__ __forceinline__ void split(float f, T& hi, T& lo) {
    hi = __float2bfloat16_rn(f);
    lo = __float2bfloat16_rn(f - __bfloat162float(hi));
  }
};

// Pipeline stage = one K chunk of every operand the passes read.  The split
// forms take 64-byte chunks (64-byte swizzle) so that four stages of A_hi,
// B_hi, A_lo, B_lo fit; the one-pass form takes 128-byte chunks.
template <int NPASS>
struct Cfg {
  static constexpr int kRowBytes = NPASS == 1 ? 128 : 64;
  static constexpr int kKSteps = kRowBytes / 32;  // MMAs of 32 bytes of K per chunk
  static constexpr int kTileA = kBM * kRowBytes;
  static constexpr int kTileB = kMaxN * kRowBytes;
  static constexpr int kStages = 4;
  static constexpr int kStage = (NPASS == 1 ? 1 : 2) * (kTileA + kTileB);
  static constexpr int kSmem = 1024 + kStages * kStage + 256;
  static __device__ __forceinline__ uint64_t desc(uint32_t saddr) {
    return NPASS == 1 ? tc::desc_sw128(saddr) : tc::desc_sw64(saddr);
  }
};

// ---- operand packing ------------------------------------------------------
// multipoles of every level l >= 2 (lexicographic boxes, FP64, nj per box) ->
// Bpar_l[sigma][Tz][Ty][Tx][JP] fp32 (tf32-rounded hi, and lo for the split);
// blockIdx.y = l - 2, levels stored back to back like the expansions.
struct LevOff {
  int64_t o[FMM_MAX_LEVELS + 1];
};

template <typename F>
__global__ void k_pack_beta(const double* __restrict__ mp, const LevOff lev_off, int nj, int JP,
                            typename F::T* __restrict__ bhi, typename F::T* __restrict__ blo) {
  const int l = blockIdx.y + 2;
  const int nl = 1 << l, H = nl >> 1;
  const unsigned tot = (unsigned)JP << (3 * l);  // boxes of the level x JP (< 2^32)
  const double* mpl = mp + lev_off.o[l] * nj;
  typename F::T* bh = bhi + lev_off.o[l] * JP;
  typename F::T* bl = blo ? blo + lev_off.o[l] * JP : nullptr;
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
    const unsigned b = e / (unsigned)JP;  // 32-bit division (JP need not be a power of two)
    const int q = (int)(e - b * (unsigned)JP);
    const int x = (int)(b & (nl - 1)), y = (int)((b >> l) & (nl - 1)), z = (int)(b >> (2 * l));
    const int sg = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2);
    const size_t dst = ((((size_t)sg * H + (z >> 1)) * H + (y >> 1)) * H + (x >> 1)) * JP + q;
    const float v = q < nj ? (float)mpl[(size_t)b * nj + q] : 0.f;
    typename F::T hi, lo;
    F::split(v, hi, lo);
    bh[dst] = hi;
    if (bl) bl[dst] = lo;
  }
}

// dense offset matrices A_h[i][q] = Ht_h[i + q] for the 343 offsets of a level:
// one block per (offset, table level); the offset's Hankel row is split into
// hi/lo once in shared memory, then expanded to the MP x JP matrix
template <int D, typename F>
__global__ void __launch_bounds__(256) k_build_tmat(PlanDev pd, const double* __restrict__ htab,
                                                    int MP, int JP,
                                                    typename F::T* __restrict__ thi,
                                                    typename F::T* __restrict__ tlo) {
  using T = typename F::T;
  const int o = blockIdx.x;
  htab += (size_t)blockIdx.y * 343 * pd.nh;
  thi += (size_t)blockIdx.y * 343 * MP * JP;
  if (tlo) tlo += (size_t)blockIdx.y * 343 * MP * JP;
  {
    int t = o;
    bool far = false;
    for (int k = 0; k < D; ++k) {
      const int hk = t % 7 - 3;
      t /= 7;
      if (hk > 1 || hk < -1) far = true;
    }
    if (!far) return;
  }
  extern __shared__ __align__(16) unsigned char smtm[];
  T* hh = reinterpret_cast<T*>(smtm);
  T* hl = hh + pd.nh;
  const double* H = htab + (size_t)o * pd.nh;
  for (int e = threadIdx.x; e < pd.nh; e += blockDim.x) F::split((float)H[e], hh[e], hl[e]);
  __syncthreads();
  const int P2 = 2 * pd.p;
  T* dh = thi + (size_t)o * MP * JP;
  T* dl = tlo ? tlo + (size_t)o * MP * JP : nullptr;
  const T zero = T(0.f);
  for (int e = threadIdx.x; e < MP * JP; e += blockDim.x) {
    const int i = e / JP, q = e - i * JP;
    T vh = zero, vl = zero;
    if (i < pd.nj && q < pd.nj) {
      const char4 a = pd.mi[i], b = pd.mi[q];
      const int m0 = a.x + b.x, m1 = a.y + b.y, m2 = a.z + b.z;
      const int idx = D == 3 ? pd.hrow[m2 * (P2 + 1) + m1] + m0 : pd.hrow[m1] + m0;
      vh = hh[idx];
      vl = hl[idx];
    }
    dh[e] = vh;
    if (dl) dl[e] = vl;
  }
}

// ---- the contraction --------------------------------------------------------
// Warp roles: warps 0-15 drain TMEM (warp w reads TMEM lanes 32(w%4).. = rows
// i, columns 64(w/4)..+63 = targets), warp 16 lane 0 issues TMA, warp 17 lane
// 0 issues MMA.  Sixteen draining warps keep the running sums at 64 floats a
// thread: 18 warps leave at most 5 per SM sub-partition, ~100 registers each.
// The tensor cores truncate when they accumulate, so a long K loop in one
// accumulator drifts; each offset's partial product therefore goes to one of
// two 256-column TMEM buffers (the whole 512 columns), and the draining warps
// add it into float registers (round-to-nearest) while the MMA warp fills the
// other buffer.
constexpr int kEpiWarps = 16;
constexpr int kNBuf = 2;
constexpr int kBufCols = kMaxN;  // TMEM columns per accumulator buffer
constexpr int kTcThreads = (kEpiWarps + 2) * 32;

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

// (sigma, delta) decode of combination c = sigma + 8 * delta_index; false if
// the offset is adjacent (not in the interaction list)
__device__ __forceinline__ bool combo(int c, int px, int py, int pz, int& sg, int& dx, int& dy,
                                      int& dz, int& hidx) {
  sg = c & 7;
  const int di = c >> 3;
  dx = di % 3 - 1;
  dy = (di / 3) % 3 - 1;
  dz = di / 9 - 1;
  const int hx = px - (sg & 1) - 2 * dx, hy = py - ((sg >> 1) & 1) - 2 * dy,
            hz = pz - ((sg >> 2) & 1) - 2 * dz;
  hidx = (hx + 3) + 7 * (hy + 3) + 49 * (hz + 3);
  return !(hx >= -1 && hx <= 1 && hy >= -1 && hy <= 1 && hz >= -1 && hz <= 1);
}

// One launch covers every level: blocks [first_block, first_block + 8 ntiles)
// of grid.x belong to level l (block = tile * 8 + pi), grid.y = 128-row block.
// The parent grid of a level is Hx x Hy x Hz cells: the whole level of a
// uniform tree (Hx = Hy = Hz = 2^(l-1), boxes lexicographic), or, for an
// adaptive tree, the window of parents spanned by the level's boxes, with
// map[(pi, cell)] the box at that position (-1: none).
// A homogeneous kernel shares one set of offset matrices over the levels, so a
// small level can ride along in the CTAs of another: its whole parent grid
// (H2^3 parents, H2 = 2^(l2-1)) is loaded into the B rows after the primary
// tile's and its targets are read off the extra MMA columns (l2 = 0: none).
// This keeps the tiny coarse levels from forming a wave of their own.
struct TcLevel {
  CUtensorMap A, Alo, B, Blo;  // offset matrices and parity-split multipoles
  CUtensorMap B2, B2lo;        // multipoles of the riding level l2
  double* lc;                  // local expansions (level base, or all boxes with map)
  double* lc2;                 // local expansions of level l2 (base)
  const int* map;              // adaptive: window cell -> box; null for uniform levels
  float scale, scale2;         // exact powers of two (shared offset matrices)
  int l, BX, BY, BZ, ntx, nty, first_block, Hx, Hy, Hz;
  int l2;
};
constexpr int kTcMaxLevels = 10;
struct TcParams {
  TcLevel lev[kTcMaxLevels];
  int nlev, nj, jchunks, MP;
  int* err;
};

template <typename F, int NPASS>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_m2l_tc(const __grid_constant__ TcParams prm) {
  int li = 0;
  while (li + 1 < prm.nlev && (int)blockIdx.x >= prm.lev[li + 1].first_block) ++li;
  const TcLevel& LV = prm.lev[li];
  const CUtensorMap* tmA = &LV.A;
  const CUtensorMap* tmAlo = &LV.Alo;
  const CUtensorMap* tmB = &LV.B;
  const CUtensorMap* tmBlo = &LV.Blo;
  const int l = LV.l, nj = prm.nj, jchunks = prm.jchunks, MP = prm.MP;
  const int BX = LV.BX, BY = LV.BY, BZ = LV.BZ, ntx = LV.ntx, nty = LV.nty;
  double* __restrict__ lc = LV.lc;
  int* __restrict__ err = prm.err;
  using C = Cfg<NPASS>;
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + C::kStages * C::kStage);
  uint64_t* empty = full + C::kStages;
  uint64_t* accf = empty + C::kStages;  // [kNBuf] accumulator filled (MMA commit)
  uint64_t* acce = accf + kNBuf;        // [kNBuf] accumulator drained (warp arrivals)
  uint64_t* drainb = acce + kNBuf;      // all MMAs of this CTA finished
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drainb + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lb = (int)blockIdx.x - LV.first_block;
  const int pi = lb & 7, mt = blockIdx.y;
  const int tile = lb >> 3;
  const int tx = tile % ntx, ty = (tile / ntx) % nty, tz = tile / (ntx * nty);
  const int X0 = tx * BX, Y0 = ty * BY, Z0 = tz * BZ;
  const int l2 = LV.l2, H2 = l2 ? 1 << (l2 - 1) : 0;
  const int N1 = BX * BY * BZ;                        // rows of the primary tile
  const int N = N1 + H2 * H2 * H2;                    // rows the TMA boxes fill
  const int Nmma = N < 16 ? 16 : (N + 15) / 16 * 16;  // MMA width; extra columns discarded
  const int nl = 1 << l, Hx = LV.Hx, Hy = LV.Hy, Hz = LV.Hz;
  const int* __restrict__ map = LV.map;
  const int px = pi & 1, py = (pi >> 1) & 1, pz = (pi >> 2) & 1;
  const uint32_t bytesA = C::kTileA, bytesB = (uint32_t)N * C::kRowBytes;
  const uint32_t stage_tx = (NPASS == 1 ? 1u : 2u) * (bytesA + bytesB);

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int bf = 0; bf < kNBuf; ++bf) {
      tc::mbar_init(&accf[bf], 1);
      tc::mbar_init(&acce[bf], kEpiWarps);
    }
    tc::mbar_init(drainb, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tslot, kBufCols * kNBuf);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;

  if (warp == kEpiWarps && lane == 0) {
    // ---------------- TMA producer ----------------
    int kk = 0;
    int last_round[C::kStages];
    for (int s = 0; s < C::kStages; ++s) last_round[s] = -1;
    bool ok = true;
    for (int c = 0; c < 216 && ok; ++c) {
      int sg, dx, dy, dz, hidx;
      if (!combo(c, px, py, pz, sg, dx, dy, dz, hidx)) continue;
      for (int ch = 0; ch < jchunks; ++ch, ++kk) {
        const int s = kk % C::kStages, r = kk / C::kStages;
        if (r > 0 && !tc::mbar_wait(&empty[s], (r - 1) & 1, err)) {
          ok = false;
          break;
        }
        unsigned char* st = sm + s * C::kStage;
        tc::mbar_expect_tx(&full[s], stage_tx);
        last_round[s] = r;
        // element offset of this K chunk (a multiple of 64 bytes)
        const int kc = ch * (C::kRowBytes / (int)sizeof(typename F::T));
        tc::tma_load_2d(st, tmA, &full[s], kc, hidx * MP + mt * kBM);
        tc::tma_load_5d(st + C::kTileA, tmB, &full[s], kc, X0 + dx, Y0 + dy, Z0 + dz, sg);
        if (l2)  // N1 is a multiple of 8 rows: the second box starts on a swizzle atom
          tc::tma_load_5d(st + C::kTileA + N1 * C::kRowBytes, &LV.B2, &full[s], kc, dx, dy, dz,
                          sg);
        if (NPASS == 3) {
          tc::tma_load_2d(st + C::kTileA + C::kTileB, tmAlo, &full[s], kc, hidx * MP + mt * kBM);
          tc::tma_load_5d(st + 2 * C::kTileA + C::kTileB, tmBlo, &full[s], kc, X0 + dx, Y0 + dy,
                          Z0 + dz, sg);
          if (l2)
            tc::tma_load_5d(st + 2 * C::kTileA + C::kTileB + N1 * C::kRowBytes, &LV.B2lo,
                            &full[s], kc, dx, dy, dz, sg);
        }
      }
    }
    if (!ok) {  // drain copies still in flight before the CTA leaves
      for (int s = 0; s < C::kStages; ++s)
        if (last_round[s] >= 0) {
          const long long t0 = clock64();
          while (!tc::mbar_try_wait(&full[s], last_round[s] & 1) &&
                 clock64() - t0 < tc::kWaitCycles) {
          }
        }
    }
  } else if (warp == kEpiWarps + 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    const uint32_t id = tc::idesc(F::kIdesc, kBM, Nmma);
    int kk = 0, g = 0;
    bool ok = true;
    for (int c = 0; c < 216 && ok; ++c) {
      int sg, dx, dy, dz, hidx;
      if (!combo(c, px, py, pz, sg, dx, dy, dz, hidx)) continue;
      const int bf = g % kNBuf;
      if (g >= kNBuf && !tc::mbar_wait(&acce[bf], ((g / kNBuf) - 1) & 1, err)) {
        ok = false;
        break;
      }
      tc::fence_after();
      const uint32_t dacc = tmem + (uint32_t)(bf * kBufCols);
      for (int ch = 0; ch < jchunks; ++ch, ++kk) {
        const int s = kk % C::kStages, r = kk / C::kStages;
        if (!tc::mbar_wait(&full[s], r & 1, err)) {
          ok = false;
          break;
        }
        tc::fence_after();
        const uint32_t st = tc::smem_u32(sm + s * C::kStage);
        const uint64_t a = C::desc(st), b = C::desc(st + C::kTileA);
        const uint64_t alo = C::desc(st + C::kTileA + C::kTileB);
        const uint64_t blo = C::desc(st + 2 * C::kTileA + C::kTileB);
#pragma unroll
        for (int k = 0; k < C::kKSteps; ++k) {
          // one MMA consumes 32 bytes of K (8 tf32 or 16 bf16) inside the swizzle atom
          const uint64_t adv = (uint64_t)(k * 32) >> 4;
          if (F::kF16) {
            tc::mma_f16(dacc, a + adv, b + adv, id, (ch | k) != 0);
            if (NPASS == 3) {
              tc::mma_f16(dacc, a + adv, blo + adv, id, 1);
              tc::mma_f16(dacc, alo + adv, b + adv, id, 1);
            }
          } else {
            tc::mma_tf32(dacc, a + adv, b + adv, id, (ch | k) != 0);
            if (NPASS == 3) {
              tc::mma_tf32(dacc, a + adv, blo + adv, id, 1);
              tc::mma_tf32(dacc, alo + adv, b + adv, id, 1);
            }
          }
        }
        tc::mma_commit(&empty[s]);
      }
      if (!ok) break;
      tc::mma_commit(&accf[bf]);
      ++g;
    }
    // the commit arrives once every MMA issued so far has finished; waiting
    // for it (time-bounded, also on the error path) means TMEM is never freed
    // under a running MMA
    tc::mma_commit(drainb);
    {
      const long long t0 = clock64();
      while (!tc::mbar_try_wait(drainb, 0) && clock64() - t0 < tc::kWaitCycles) {
      }
    }
  } else if (warp < kEpiWarps) {
    // ---------------- drain TMEM into float registers ----------------
    constexpr int kCols = kMaxN / (kEpiWarps / 4);       // columns per draining warp
    const int quad = warp & 3, c0 = (warp >> 2) * kCols;  // TMEM lanes / first column
    float sum[kCols];
#pragma unroll
    for (int j = 0; j < kCols; ++j) sum[j] = 0.f;
    bool ok = true;
    int g = 0;
    for (int c = 0; c < 216; ++c) {
      int sg, dx, dy, dz, hidx;
      if (!combo(c, px, py, pz, sg, dx, dy, dz, hidx)) continue;
      const int bf = g % kNBuf;
      if (!tc::mbar_wait(&accf[bf], (g / kNBuf) & 1, err)) {
        ok = false;
        break;
      }
      tc::fence_after();
      const uint32_t base =
          tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(bf * kBufCols + c0);
      // groups of 16 columns, each loaded then summed (16 registers in flight)
#pragma unroll
      for (int gq = 0; gq < kCols / 16; ++gq) {
        if (c0 + 16 * gq < N) {
          uint32_t r0[16];
          tc::tmem_ld16_nowait(base + (uint32_t)(16 * gq), r0);
          tc::tmem_wait();
#pragma unroll
          for (int j = 0; j < 16; ++j) sum[16 * gq + j] += __uint_as_float(r0[j]);
        }
      }
      tc::fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[bf]);
      ++g;
    }
    ok = ok && !(*(volatile int*)err & 2);
    if (ok) {
      const int i = mt * kBM + quad * 32 + lane;
#pragma unroll
      for (int jn = 0; jn < kCols; ++jn) {
        const int n = c0 + jn;
        const float sv = sum[jn];
        if (n < N1) {
          const int x = X0 + n % BX, y = Y0 + (n / BX) % BY, z = Z0 + n / (BX * BY);
          if (x < Hx && y < Hy && z < Hz && i < nj) {
            const int64_t t =
                map ? (int64_t)map[(((size_t)pi * Hz + z) * Hy + y) * Hx + x]
                    : ((int64_t)(2 * z + pz) * nl + (2 * y + py)) * nl + (2 * x + px);
            if (t >= 0) lc[t * nj + i] += (double)(sv * LV.scale);
          }
        } else if (n < N && i < nj) {  // the riding level's targets
          const int n2 = n - N1, nl2 = 2 * H2;
          const int x = n2 % H2, y = (n2 / H2) % H2, z = n2 / (H2 * H2);
          const int64_t t = ((int64_t)(2 * z + pz) * nl2 + (2 * y + py)) * nl2 + (2 * x + px);
          LV.lc2[t * nj + i] += (double)(sv * LV.scale2);
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kBufCols * kNBuf);
}

// ---- host side: tensor maps ---------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

bool make_map(CUtensorMap* m, void* base, int rank, const cuuint64_t* dims,
              const cuuint64_t* strides, const cuuint32_t* box, CUtensorMapDataType dt,
              int row_bytes) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  return fn(m, dt, (cuuint32_t)rank, base, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE,
            row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// Target tile of a parent grid Hx x Hy x Hz: up to 16 x 4 x 4 (or 8 x 8 x 4)
// = 256 parents, x fastest.
void tile_shape(int Hx, int Hy, int Hz, TcLevel* v) {
  v->BX = std::min(16, Hx);
  v->BZ = std::min(4, Hz);
  v->BY = std::min(Hy, kMaxN / (v->BX * v->BZ));
  v->ntx = (Hx + v->BX - 1) / v->BX;
  v->nty = (Hy + v->BY - 1) / v->BY;
}

// offset matrices A_h (hi and lo) of a uniform tree from the derivative tables
template <typename F, int NPASS>
void build_tables(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st) {
  using T = typename F::T;
  const PlanDev& pd = P->pd;
  const bool shared_t = pd.kernel != FMM_KERNEL_YUKAWA;  // homogeneous G
  const int tlev = shared_t ? 1 : (P->desc.levels - 1);
  T* thi0 = static_cast<T*>(ws.tc_tmat[0]);
  T* tlo = NPASS == 3 ? static_cast<T*>(ws.tc_tmat[1]) : nullptr;
  const size_t sm = 2 * sizeof(T) * pd.nh;
  if (sm > 48 * 1024)
    cudaFuncSetAttribute(k_build_tmat<3, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_build_tmat<3, F><<<dim3(343, tlev), 256, sm, st>>>(pd, ws.htab, ws.tc_mp, ws.tc_jp, thi0, tlo);
}

template <typename F, int NPASS>
cudaError_t run_all_levels(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st,
                           bool tables_ready) {
  using C = Cfg<NPASS>;
  const PlanDev& pd = P->pd;
  const int L = P->desc.levels;
  const int nj = pd.nj, JP = ws.tc_jp, MP = ws.tc_mp;
  const int noff = 343;
  const bool shared_t = pd.kernel != FMM_KERNEL_YUKAWA;  // homogeneous G
  const int tlev = shared_t ? 1 : (L - 1);
  using T = typename F::T;
  const size_t esz = sizeof(T);
  const CUtensorMapDataType dt =
      F::kF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  T* bhi0 = static_cast<T*>(ws.tc_bpar[0]);
  T* thi0 = static_cast<T*>(ws.tc_tmat[0]);
  T* blo = NPASS == 3 ? static_cast<T*>(ws.tc_bpar[1]) : nullptr;
  T* tlo = NPASS == 3 ? static_cast<T*>(ws.tc_tmat[1]) : nullptr;
  LevOff lo;
  for (int l = 0; l <= FMM_MAX_LEVELS; ++l) lo.o[l] = l <= L + 1 ? ws.lev_off[l] : 0;
  k_pack_beta<F><<<dim3(152 * 4, L - 1), 256, 0, st>>>(ws.mp, lo, nj, JP, bhi0, blo);
  if (!tables_ready) build_tables<F, NPASS>(P, ws, st);
  TcParams prm;
  std::memset(&prm, 0, sizeof(prm));
  prm.nj = nj;
  const int row = C::kRowBytes / (int)esz;  // elements per K chunk
  prm.jchunks = JP / row;
  prm.MP = MP;
  prm.err = &ws.geom->flag;
  int nb = 0;
  // largest level first: its tiles start earliest; with shared offset
  // matrices level 2 rides along in level 3's CTAs
  const int lmin = (shared_t && L >= 3) ? 3 : 2;
  for (int l = L; l >= lmin; --l) {
    TcLevel& v = prm.lev[prm.nlev++];
    const int nl = 1 << l, H = nl >> 1;
    v.l = l;
    v.l2 = 0;
    tile_shape(H, H, H, &v);
    const int ntz = (H + v.BZ - 1) / v.BZ;
    v.first_block = nb;
    nb += v.ntx * v.nty * ntz * 8;
    v.lc = ws.lc + ws.lev_off[l] * nj;
    v.map = nullptr;
    v.Hx = v.Hy = v.Hz = H;
    const int ti = shared_t ? 0 : l - 2;
    T* th = thi0 + (size_t)ti * noff * MP * JP;
    T* bh = bhi0 + ws.lev_off[l] * JP;
    v.scale = 1.0f;
    if (shared_t) {  // Ht_l = Ht_2 * (s_2/s_l)^{-deg}: deg -1 (Laplace), +1 (biharmonic)
      const int k = l - 2;
      v.scale = pd.kernel == FMM_KERNEL_LAPLACE ? std::ldexp(1.0f, k) : std::ldexp(1.0f, -k);
    }
    cuuint64_t dA[2] = {(cuuint64_t)JP, (cuuint64_t)noff * MP};
    cuuint64_t sA[1] = {(cuuint64_t)JP * esz};
    cuuint32_t bA[2] = {(cuuint32_t)row, (cuuint32_t)kBM};
    cuuint64_t dB[5] = {(cuuint64_t)JP, (cuuint64_t)H, (cuuint64_t)H, (cuuint64_t)H, 8};
    cuuint64_t sB[4] = {(cuuint64_t)JP * esz, (cuuint64_t)JP * esz * H,
                        (cuuint64_t)JP * esz * H * H, (cuuint64_t)JP * esz * H * H * H};
    cuuint32_t bB[5] = {(cuuint32_t)row, (cuuint32_t)v.BX, (cuuint32_t)v.BY, (cuuint32_t)v.BZ, 1};
    const int rb = C::kRowBytes;
    if (!make_map(&v.A, th, 2, dA, sA, bA, dt, rb)) return cudaErrorInvalidValue;
    if (!make_map(&v.B, bh, 5, dB, sB, bB, dt, rb)) return cudaErrorInvalidValue;
    v.Alo = v.A;
    v.Blo = v.B;
    if (NPASS == 3) {
      if (!make_map(&v.Alo, tlo + (size_t)ti * noff * MP * JP, 2, dA, sA, bA, dt, rb))
        return cudaErrorInvalidValue;
      if (!make_map(&v.Blo, blo + ws.lev_off[l] * JP, 5, dB, sB, bB, dt, rb))
        return cudaErrorInvalidValue;
    }
    if (l == 3 && lmin == 3) {  // level 2: 2 x 2 x 2 parents after level 3's 64
      v.l2 = 2;
      v.lc2 = ws.lc + ws.lev_off[2] * nj;
      v.scale2 = 1.0f;
      cuuint64_t d2[5] = {(cuuint64_t)JP, 2, 2, 2, 8};
      cuuint64_t s2[4] = {(cuuint64_t)JP * esz, (cuuint64_t)JP * esz * 2,
                          (cuuint64_t)JP * esz * 4, (cuuint64_t)JP * esz * 8};
      cuuint32_t b2[5] = {(cuuint32_t)row, 2, 2, 2, 1};
      if (!make_map(&v.B2, bhi0 + ws.lev_off[2] * JP, 5, d2, s2, b2, dt, rb))
        return cudaErrorInvalidValue;
      v.B2lo = v.B2;
      if (NPASS == 3 &&
          !make_map(&v.B2lo, blo + ws.lev_off[2] * JP, 5, d2, s2, b2, dt, rb))
        return cudaErrorInvalidValue;
    }
  }
  // per call: the attribute belongs to the current device's context
  cudaFuncSetAttribute(k_m2l_tc<F, NPASS>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
  mark_contraction(P, 0, st);
  k_m2l_tc<F, NPASS><<<dim3(nb, MP / kBM), kTcThreads, C::kSmem, st>>>(prm);
  mark_contraction(P, 1, st);
  return cudaGetLastError();
}

// ---- adaptive trees: every level packed into a dense window ----------------
// bounds[6 l + k] / [6 l + 3 + k]: smallest / largest coordinate k of the
// boxes of level l
__global__ void k_alevel_bounds_init(int* bounds, int n) {
  const int i = threadIdx.x;
  if (i < n) bounds[i] = (i % 6) < 3 ? 0x7fffffff : -1;
}

__global__ void k_alevel_bounds(ATree t, int* __restrict__ bounds) {
  const int b = t.loff[2] + blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= t.loff[t.maxlev + 1]) return;
  int l, c[3];
  abox(t, b, &l, c);
  for (int k = 0; k < 3; ++k) {
    atomicMin(&bounds[6 * l + k], c[k]);
    atomicMax(&bounds[6 * l + 3 + k], c[k]);
  }
}

// the level's boxes into Bpar[sigma][Tz][Ty][Tx][JP] (hi and lo) of a window
// with parent origin W and size H, and map[sigma][Tz][Ty][Tx] = box
template <typename F>
__global__ void k_apack(ATree t, int l, const double* __restrict__ mp, int nj, int JP, int W0x,
                        int W0y, int W0z, int Hx, int Hy, int Hz, typename F::T* __restrict__ bhi,
                        typename F::T* __restrict__ blo, int* __restrict__ map) {
  const int b0 = t.loff[l];
  const unsigned tot = (unsigned)(t.loff[l + 1] - b0) * (unsigned)JP;
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
    const unsigned bi = e / (unsigned)JP;
    const int q = (int)(e - bi * (unsigned)JP);
    const int b = b0 + (int)bi;
    int c[3];
    demorton3(t.key[b], l, c);
    const int sg = (c[0] & 1) | ((c[1] & 1) << 1) | ((c[2] & 1) << 2);
    const size_t cell =
        (((size_t)sg * Hz + ((c[2] >> 1) - W0z)) * Hy + ((c[1] >> 1) - W0y)) * Hx + ((c[0] >> 1) - W0x);
    const float v = q < nj ? (float)mp[(size_t)b * nj + q] : 0.f;
    typename F::T hi, lo;
    F::split(v, hi, lo);
    bhi[cell * JP + q] = hi;
    if (blo) blo[cell * JP + q] = lo;
    if (q == 0) map[cell] = b;
  }
}

template <typename F, int NPASS>
cudaError_t run_adaptive(const fmm_plan_s* P, const Workspace& ws, const ATree& t,
                         cudaStream_t st, int* nl, unsigned* done) {
  using C = Cfg<NPASS>;
  using T = typename F::T;
  const PlanDev& pd = P->pd;
  const int nj = pd.nj, JP = ws.tc_jp, MP = ws.tc_mp;
  const int noff = 343;
  const bool shared_t = pd.kernel != FMM_KERNEL_YUKAWA;  // homogeneous G
  const int tlev = shared_t ? 1 : (t.maxlev - 1);
  const size_t esz = sizeof(T);
  const CUtensorMapDataType dt =
      F::kF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  T* thi0 = static_cast<T*>(ws.tc_tmat[0]);
  T* tlo = NPASS == 3 ? static_cast<T*>(ws.tc_tmat[1]) : nullptr;
  // coordinate bounds of every level (one synchronisation)
  const int nbnd = 6 * (t.maxlev + 1);
  k_alevel_bounds_init<<<1, 128, 0, st>>>(ws.tc_bounds, nbnd);
  const int nbox2 = t.loff[t.maxlev + 1] - t.loff[2];
  k_alevel_bounds<<<(nbox2 + 255) / 256, 256, 0, st>>>(t, ws.tc_bounds);
  *nl += 2;
  int bnd[6 * (FMM_MAX_ADEPTH + 2)];
  cudaMemcpyAsync(bnd, ws.tc_bounds, sizeof(int) * nbnd, cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  {
    const size_t sm = 2 * sizeof(T) * pd.nh;
    if (sm > 48 * 1024)
      cudaFuncSetAttribute(k_build_tmat<3, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_build_tmat<3, F><<<dim3(noff, tlev), 256, sm, st>>>(pd, ws.htab, MP, JP, thi0, tlo);
    ++*nl;
  }
  TcParams prm;
  std::memset(&prm, 0, sizeof(prm));
  prm.nj = nj;
  const int row = C::kRowBytes / (int)esz;  // elements per K chunk
  prm.jchunks = JP / row;
  prm.MP = MP;
  prm.err = &ws.geom->flag;
  int nb = 0;
  char* arena = static_cast<char*>(ws.tc_arena);
  size_t used = 0;
  const size_t cell_bytes = (size_t)JP * esz;
  for (int l = t.maxlev; l >= 2; --l) {  // largest (finest) level first
    if (bnd[6 * l + 3] < 0) continue;    // no box at this level
    int W0[3], H[3];
    for (int k = 0; k < 3; ++k) {
      W0[k] = bnd[6 * l + k] >> 1;
      H[k] = (bnd[6 * l + 3 + k] >> 1) - W0[k] + 1;
    }
    const size_t cells = (size_t)8 * H[0] * H[1] * H[2];
    auto a256 = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t need = a256(cells * cell_bytes) * (NPASS == 3 ? 2 : 1) + a256(cells * sizeof(int));
    if (used + need > ws.tc_arena_bytes) continue;  // left to the CUDA cores
    T* bhi = reinterpret_cast<T*>(arena + used);
    T* blo = NPASS == 3 ? reinterpret_cast<T*>(arena + used + a256(cells * cell_bytes)) : nullptr;
    int* map = reinterpret_cast<int*>(arena + used + a256(cells * cell_bytes) * (NPASS == 3 ? 2 : 1));
    used += need;
    cudaMemsetAsync(bhi, 0, cells * cell_bytes, st);
    if (blo) cudaMemsetAsync(blo, 0, cells * cell_bytes, st);
    cudaMemsetAsync(map, 0xff, cells * sizeof(int), st);
    const unsigned nbl = (unsigned)(t.loff[l + 1] - t.loff[l]);
    k_apack<F><<<std::min<unsigned>((nbl * JP + 255) / 256, 152 * 8), 256, 0, st>>>(
        t, l, ws.mp, nj, JP, W0[0], W0[1], W0[2], H[0], H[1], H[2], bhi, blo, map);
    ++*nl;
    TcLevel& v = prm.lev[prm.nlev++];
    v.l = l;
    v.l2 = 0;
    v.Hx = H[0];
    v.Hy = H[1];
    v.Hz = H[2];
    tile_shape(H[0], H[1], H[2], &v);
    const int ntz = (H[2] + v.BZ - 1) / v.BZ;
    v.first_block = nb;
    nb += v.ntx * v.nty * ntz * 8;
    v.lc = ws.lc;
    v.map = map;
    const int ti = shared_t ? 0 : l - 2;
    v.scale = 1.0f;
    if (shared_t) {
      const int k = l - 2;
      v.scale = pd.kernel == FMM_KERNEL_LAPLACE ? std::ldexp(1.0f, k) : std::ldexp(1.0f, -k);
    }
    cuuint64_t dA[2] = {(cuuint64_t)JP, (cuuint64_t)noff * MP};
    cuuint64_t sA[1] = {(cuuint64_t)JP * esz};
    cuuint32_t bA[2] = {(cuuint32_t)row, (cuuint32_t)kBM};
    cuuint64_t dB[5] = {(cuuint64_t)JP, (cuuint64_t)H[0], (cuuint64_t)H[1], (cuuint64_t)H[2], 8};
    cuuint64_t sB[4] = {(cuuint64_t)JP * esz, (cuuint64_t)JP * esz * H[0],
                        (cuuint64_t)JP * esz * H[0] * H[1],
                        (cuuint64_t)JP * esz * H[0] * H[1] * H[2]};
    cuuint32_t bB[5] = {(cuuint32_t)row, (cuuint32_t)v.BX, (cuuint32_t)v.BY, (cuuint32_t)v.BZ, 1};
    const int rb = C::kRowBytes;
    if (!make_map(&v.A, thi0 + (size_t)ti * noff * MP * JP, 2, dA, sA, bA, dt, rb))
      return cudaErrorInvalidValue;
    if (!make_map(&v.B, bhi, 5, dB, sB, bB, dt, rb)) return cudaErrorInvalidValue;
    v.Alo = v.A;
    v.Blo = v.B;
    if (NPASS == 3) {
      if (!make_map(&v.Alo, tlo + (size_t)ti * noff * MP * JP, 2, dA, sA, bA, dt, rb))
        return cudaErrorInvalidValue;
      if (!make_map(&v.Blo, blo, 5, dB, sB, bB, dt, rb)) return cudaErrorInvalidValue;
    }
    *done |= 1u << l;
    if (prm.nlev == kTcMaxLevels) break;
  }
  if (prm.nlev == 0) return cudaGetLastError();
  cudaFuncSetAttribute(k_m2l_tc<F, NPASS>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
  k_m2l_tc<F, NPASS><<<dim3(nb, MP / kBM), kTcThreads, C::kSmem, st>>>(prm);
  ++*nl;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_m2l_tc(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st, int* nl,
                          bool tables_ready) {
  const int L = P->desc.levels;
  if (P->pd.d != 3) return launch_m2l_simt_levels(P, ws, 2, L, st, nl);
  const int prec = P->desc.precision;
  const cudaError_t e =
      prec == FMM_PREC_BF16X3   ? run_all_levels<FmtBF16, 3>(P, ws, st, tables_ready)
      : prec == FMM_PREC_TF32X3 ? run_all_levels<FmtTF32, 3>(P, ws, st, tables_ready)
                                : run_all_levels<FmtTF32, 1>(P, ws, st, tables_ready);
  *nl += tables_ready ? 2 : 3;
  return e;
}

// the offset matrices alone (uniform 3D tree, tensor-core precisions), so
// that they can be built on another stream ahead of the contraction
cudaError_t launch_m2l_tc_tables(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st,
                                 int* nl) {
  const int prec = P->desc.precision;
  if (prec == FMM_PREC_BF16X3) build_tables<FmtBF16, 3>(P, ws, st);
  else if (prec == FMM_PREC_TF32X3) build_tables<FmtTF32, 3>(P, ws, st);
  else build_tables<FmtTF32, 1>(P, ws, st);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_adaptive_m2l_tc(const fmm_plan_s* P, const Workspace& ws, const ATree& t,
                                   cudaStream_t st, int* nl, unsigned* done) {
  *done = 0;
  if (t.maxlev < 2) return cudaGetLastError();
  const int prec = P->desc.precision;
  return prec == FMM_PREC_BF16X3   ? run_adaptive<FmtBF16, 3>(P, ws, t, st, nl, done)
         : prec == FMM_PREC_TF32X3 ? run_adaptive<FmtTF32, 3>(P, ws, t, st, nl, done)
                                   : run_adaptive<FmtTF32, 1>(P, ws, t, st, nl, done);
}
