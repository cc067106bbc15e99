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
// outside the domain) is a dense operand, and so is the offset matrix
//   A_h[i][q] = Ht_h[i + q]   (i, q in j).
//
// Orientation.  The MMA's M dimension (the 128 TMEM lanes) holds 128 target
// parents, N holds the local coefficients i and K the multipole
// coefficients q:
//   D[T][i] += sum_q Bpar[sigma][T + delta][q] * A_h[i][q],
// so |j| is padded only to the MMA's N granularity of 16 (130 -> 144 for the
// biharmonic kernel at p = 8) and the K steps that hold nothing but padding
// are not issued.  Above 256 columns |j| is split into column blocks (one per
// grid row); where one block leaves room, the offset matrices of 2, 4 or 8
// child classes pi are stacked along N (one MMA of up to 256 columns), so small
// |j| still run the long MMAs the tensor pipe needs (3D Laplace p = 10:
// |j| = 121 -> two classes of 128 columns).  A CTA runs every (sigma, delta)
// that is an interaction for at least one of its classes; an offset that is
// adjacent for one class meets that class's zero matrix.
//
// Precision: TF32 (one pass), or TF32x3 / BF16x3 (a = a_hi + a_lo split,
// three passes a_hi b_hi + a_hi b_lo + a_lo b_hi), FP32 accumulation.
#include <algorithm>
#include <cstring>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "adaptive.cuh"
#include "expansions.cuh"
#include "tc_ptx.cuh"

cudaError_t launch_m2l_simt_levels(const fmm_plan_s* P, const Workspace& ws, int l0, int l1,
                                   cudaStream_t st, int* nl);

namespace {

constexpr int kBM = 128;       // target parents per CTA = MMA M = TMEM lanes
constexpr int kMaxN = 256;     // MMA N: columns of i (times stacked classes)
constexpr int kMaxStages = 8;  // pipeline depth bound
constexpr int kSmemCap = 227 * 1024;  // opt-in shared memory per CTA

// Operand formats: tf32 (fp32 storage, kind::tf32) and bf16 (kind::f16).  Both
// split a value into hi + lo.  The split works on the float rounding of the
// value (one conversion from FP64): lo = f - hi is exact in float, and keeps
// the bits the tf32/bf16 format drops from hi.
struct FmtTF32 {
  using T = float;
  static constexpr int kIdesc = 2;
  static constexpr bool kF16 = false;
  static constexpr bool kScaled = false;
  static constexpr CUtensorMapDataType kMapType = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  static __device__ __forceinline__ void split(float f, T& hi, T& lo) {
    const float h = tc::tf32_rna(f);
    hi = h;
    lo = tc::tf32_rna(f - h);
  }
};
struct FmtBF16 {
  using T = __nv_bfloat16;
  static constexpr int kIdesc = 1;
  static constexpr bool kF16 = true;
  static constexpr bool kScaled = false;
  static constexpr CUtensorMapDataType kMapType = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  static __device__ __forceinline__ void split(float f, T& hi, T& lo) {
    hi = __float2bfloat16_rn(f);
    lo = __float2bfloat16_rn(f - __bfloat162float(hi));
  }
};
// fp16 (kind::f16, type 0): tf32's 11-bit significand, a 5-bit exponent.
// The operands are scaled into its range (kScaled).  With S_m = m! (sqrt 2)^|m|
// (the float table fact_f): a box's multipole bt_q S_q, times 2^-e_box so that
// its largest entry lies in [1/2, 1); the offset matrix Ht_{i+q} / (S_i S_q)
// over the power of two of the level's derivative scale.  Dividing by i! q!
// turns the Hankel entries into binomially weighted Taylor coefficients of G,
// which grow like (sqrt 2)^{|i+q|} at the nearest offsets (their singularity
// lies sqrt 2 box sides away in complex directions); (sqrt 2)^{|i+q|} takes
// that growth out, so the entries stay below ~10 up to p = 16 (65504 is
// fp16's largest) while the rows of high |i| stay out of the subnormal range.
// The draining warps multiply each offset's product by 2^e_box of the row's
// source box and the epilogue by S_i and the table scale.
struct FmtF16 {
  using T = __half;
  static constexpr int kIdesc = 0;
  static constexpr bool kF16 = true;
  static constexpr bool kScaled = true;
  static constexpr CUtensorMapDataType kMapType = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  static __device__ __forceinline__ void split(float f, T& hi, T& lo) {
    hi = __float2half_rn(f);
    lo = __float2half_rn(f - __half2float(hi));
  }
};

// the power of two of the derivative tables' scale at level l (Laplace
// 1/(4 pi s), biharmonic s, the screened and oscillatory kernels 1/s): the
// F16X3 offset matrices are divided by it
__host__ __device__ inline double tc_norm(int kernel, double size, int l) {
  const double s = size / (double)(1 << l);
  const double ds = kernel == FMM_KERNEL_LAPLACE ? 1.0 / (4.0 * 3.14159265358979323846 * s)
                    : kernel == FMM_KERNEL_BIHARMONIC ? s
                                                      : 1.0 / s;
  return std::ldexp(1.0, std::ilogb(ds));
}

// A pipeline stage holds one K chunk of every operand the passes read:
// [sources hi | offset matrices hi | sources lo | offset matrices lo], in
// 128-byte chunks (128-byte swizzle); the row bytes must match tc_shape().
// Each stage feeds 4 K steps (12 MMAs in the split forms) per barrier round:
// measured on GB300, 64-byte chunks (twice the rounds) ran the contraction
// 15-18% slower (biharmonic p = 8, L = 6: 11.9 against 10.1 ms, TF32x3).
template <int NPASS>
struct Cfg {
  static constexpr int kRowBytes = 128;
  static constexpr int kKSteps = kRowBytes / 32;  // MMAs of 32 bytes of K per chunk
  static constexpr int kTileS = kBM * kRowBytes;  // the source tile (MMA A)
  static constexpr int kHalves = NPASS == 1 ? 1 : 2;
  static __device__ __forceinline__ uint64_t desc(uint32_t saddr) { return tc::desc_sw128(saddr); }
  // bytes of one stage for an N of ntot columns
  static __host__ __device__ int stage_bytes(int ntot) {
    return kHalves * (kTileS + ntot * kRowBytes);
  }
};

// ---- operand packing ------------------------------------------------------
// multipoles of every level l >= 2 (lexicographic boxes, FP64, nj per box) ->
// Bpar_l[sigma][Tz][Ty][Tx][JP] (hi, and lo for the split);
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

// The F16X3 packing: one warp per box, bt_q S_q scaled by 2^-e so that its
// largest entry lies in [1/2, 1); 2^e goes to bscale in the same parity-split
// cell order (one value per box).
template <typename F>
__global__ void __launch_bounds__(256) k_pack_beta_scaled(const double* __restrict__ mp,
                                                          const LevOff lev_off, int nj, int JP,
                                                          const float* __restrict__ fact_f,
                                                          typename F::T* __restrict__ bhi,
                                                          typename F::T* __restrict__ blo,
                                                          float* __restrict__ bscale) {
  const int l = blockIdx.y + 2;
  const int nl = 1 << l, H = nl >> 1;
  const int64_t nbox = (int64_t)1 << (3 * l);
  const double* mpl = mp + lev_off.o[l] * nj;
  typename F::T* bh = bhi + lev_off.o[l] * JP;
  typename F::T* bl = blo + lev_off.o[l] * JP;
  float* bs = bscale + lev_off.o[l];
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nbox; b += nw) {
    const int x = (int)(b & (nl - 1)), y = (int)((b >> l) & (nl - 1)), z = (int)(b >> (2 * l));
    const int sg = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2);
    const size_t cell = (((size_t)sg * H + (z >> 1)) * H + (y >> 1)) * H + (x >> 1);
    const double* src = mpl + b * nj;
    float m = 0.f;
    for (int q = lane; q < nj; q += 32) m = fmaxf(m, fabsf((float)src[q] * fact_f[q]));
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    const int e = m > 0.f ? ilogbf(m) + 1 : 0;
    const float down = ldexpf(1.f, -e);  // exact
    for (int q = lane; q < JP; q += 32) {
      const float v = q < nj ? (float)src[q] * fact_f[q] * down : 0.f;
      typename F::T hi, lo;
      F::split(v, hi, lo);
      bh[cell * JP + q] = hi;
      bl[cell * JP + q] = lo;
    }
    if (lane == 0) bs[cell] = ldexpf(1.f, e);
  }
}

// dense offset matrices A_h[i][q] = Ht_h[i + q] (rows i < NPT, columns q < JP,
// zero outside j) for the 343 offsets of a level: one block per (offset,
// table level).  The offsets of adjacent boxes get zero matrices: a CTA that
// serves several child classes meets them for the classes the offset is not
// an interaction of.  The offset's Hankel row is split into hi/lo once in
// shared memory, then expanded.
template <int D, typename F>
__global__ void __launch_bounds__(256) k_build_tmat(PlanDev pd, const Geom* __restrict__ g,
                                                    const double* __restrict__ htab,
                                                    int NPT, int JP,
                                                    typename F::T* __restrict__ thi,
                                                    typename F::T* __restrict__ tlo) {
  using T = typename F::T;
  const int o = blockIdx.x;
  htab += (size_t)blockIdx.y * 343 * pd.nh;
  thi += (size_t)blockIdx.y * 343 * NPT * JP;
  if (tlo) tlo += (size_t)blockIdx.y * 343 * NPT * JP;
  bool far = false;
  {
    int t = o;
    for (int k = 0; k < D; ++k) {
      const int hk = t % 7 - 3;
      t /= 7;
      if (hk > 1 || hk < -1) far = true;
    }
  }
  T* dh = thi + (size_t)o * NPT * JP;
  T* dl = tlo ? tlo + (size_t)o * NPT * JP : nullptr;
  const T zero = T(0.f);
  if (!far) {
    for (int e = threadIdx.x; e < NPT * JP; e += blockDim.x) {
      dh[e] = zero;
      if (dl) dl[e] = zero;
    }
    return;
  }
  extern __shared__ __align__(16) unsigned char smtm[];
  const double* H = htab + (size_t)o * pd.nh;
  const int P2 = 2 * pd.p;
  if (F::kScaled) {  // Ht_{i+q} / (S_i S_q norm), with the very float S_m the packing uses
    double* rf = reinterpret_cast<double*>(smtm);  // 1 / S_m of the stored set
    for (int e = threadIdx.x; e < pd.nj; e += blockDim.x) rf[e] = 1.0 / (double)pd.fact_f[e];
    __syncthreads();
    const double rn = 1.0 / tc_norm(pd.kernel, g->size, blockIdx.y + 2);  // a power of two
    for (int e = threadIdx.x; e < NPT * JP; e += blockDim.x) {
      const int i = e / JP, q = e - i * JP;
      T vh = zero, vl = zero;
      if (i < pd.nj && q < pd.nj) {
        const char4 a = pd.mi[i], b = pd.mi[q];
        const int m0 = a.x + b.x, m1 = a.y + b.y, m2 = a.z + b.z;
        const int idx = D == 3 ? pd.hrow[m2 * (P2 + 1) + m1] + m0 : pd.hrow[m1] + m0;
        F::split((float)(H[idx] * rn * rf[i] * rf[q]), vh, vl);
      }
      dh[e] = vh;
      if (dl) dl[e] = vl;
    }
    return;
  }
  T* hh = reinterpret_cast<T*>(smtm);
  T* hl = hh + pd.nh;
  for (int e = threadIdx.x; e < pd.nh; e += blockDim.x) F::split((float)H[e], hh[e], hl[e]);
  __syncthreads();
  for (int e = threadIdx.x; e < NPT * JP; e += blockDim.x) {
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
// Warp roles: warps 0-15 drain TMEM (warp w reads TMEM lanes 32(w%4).. =
// target parents, and a quarter of the columns), warp 16 lane 0 issues TMA,
// warp 17 lane 0 issues MMA.  Eighteen warps put five on an SM sub-partition,
// which caps a thread at 96 registers: the drain's 64 running sums fit, and
// the MMA loop must stay lean (a spilled loop variable there cost 15%).  The tensor cores truncate when they accumulate,
// so a long K loop in one accumulator drifts; each offset's partial product
// therefore goes to one of two 256-column TMEM buffers (the whole 512
// columns), and the draining warps add it into float registers
// (round-to-nearest) while the MMA warp fills the other buffer.  At the end
// the sums go through shared memory so that the FP64 local expansions are
// written row by row (coalesced).
constexpr int kEpiWarps = 16;
constexpr int kNBuf = 2;         // accumulator buffers of 256 columns
constexpr int kTmemCols = 512;   // the whole tensor memory of the SM
constexpr int kTcThreads = (kEpiWarps + 2) * 32;
// running sums per thread: a quarter of the MMA's columns; instantiated for
// N <= 192 (48) and N <= 256 (64) -- the smaller count leaves the registers
// that the F16X3 drain's row scales need under the 96-register cap
constexpr int kColsSmall = 48;
constexpr int kColsLarge = kMaxN / (kEpiWarps / 4);

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}
// barrier of the 16 draining warps alone (the TMA and MMA threads go their way)
__device__ __forceinline__ void drain_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kEpiWarps * 32) : "memory");
}

// Combination c = sigma + 8 * delta_index of a source child and a parent shift.
struct Combo {
  int sg, dx, dy, dz;
};
__device__ __forceinline__ Combo combo(int c) {
  Combo k;
  k.sg = c & 7;
  const int di = c >> 3;
  k.dx = di % 3 - 1;
  k.dy = (di / 3) % 3 - 1;
  k.dz = di / 9 - 1;
  return k;
}
// offset index (0..342) of combination k for targets of class pi; *far is
// false when the offset is adjacent (not in the interaction list)
__device__ __forceinline__ int offset_of(const Combo& k, int pi, bool* far) {
  const int hx = (pi & 1) - (k.sg & 1) - 2 * k.dx;
  const int hy = ((pi >> 1) & 1) - ((k.sg >> 1) & 1) - 2 * k.dy;
  const int hz = ((pi >> 2) & 1) - ((k.sg >> 2) & 1) - 2 * k.dz;
  *far = !(hx >= -1 && hx <= 1 && hy >= -1 && hy <= 1 && hz >= -1 && hz <= 1);
  return (hx + 3) + 7 * (hy + 3) + 49 * (hz + 3);
}
// the combination is an interaction for at least one of the classes pi0..
__device__ __forceinline__ bool any_far(const Combo& k, int pi0, int ncls) {
  bool any = false;
  for (int u = 0; u < ncls; ++u) {
    bool f;
    offset_of(k, pi0 + u, &f);
    any |= f;
  }
  return any;
}

// One launch covers every level: blocks [first_block, first_block + ntiles *
// 8 / ncls) of grid.x belong to level l (block = tile * (8 / ncls) + class
// group), grid.y = column block of i.
// The parent grid of a level is Hx x Hy x Hz cells: the whole level of a
// uniform tree (Hx = Hy = Hz = 2^(l-1), boxes lexicographic), or, for an
// adaptive tree, the window of parents spanned by the level's boxes, with
// map[(pi, cell)] the box at that position (-1: none).
// A homogeneous kernel shares one set of offset matrices over the levels, so a
// small level can ride along in the CTAs of another: its whole parent grid
// (H2^3 parents, H2 = 2^(l2-1)) is loaded into the source rows after the
// primary tile's and its targets are read off the extra TMEM lanes (l2 = 0:
// none).  This keeps the tiny coarse levels from forming a wave of their own.
// Gathered levels (adaptive trees, gather != 0): the MMA's 128 rows are 128
// target cells of one class taken from a list (tlist: the cells holding a box
// with targets, grouped by class at offsets toff[0..8], Morton order inside a
// class), and each offset's source rows are gathered from the parity-split
// window (rows ghi, glo; row zero_row is all zeros and stands for a source
// outside the window) by the producer warp's cp.async copies into the layout
// the TMA would have written.  CTA 8k + u of the level takes entries
// 128k .. 128k + 127 of class u's list: the k-th chunks of the eight classes
// cover about the same region and run together, so the window rows they share
// are read from L2 (class-major order measured 2.7x slower per CTA, the
// window exceeding L2); CTAs past a class's list leave at once.
struct TcLevel {
  CUtensorMap S, Slo;    // parity-split multipoles of the level (MMA A)
  CUtensorMap S2, S2lo;  // multipoles of the riding level l2
  CUtensorMap H, Hlo;    // offset matrices of the level (MMA B)
  double* lc;            // local expansions (level base, or all boxes with map)
  double* lc2;           // local expansions of level l2 (base)
  const int* map;        // adaptive: window cell -> box; null for uniform levels
  const float* bscale;   // F16X3: 2^e_box of the level's packed multipoles (cell order)
  const float* bscale2;  // the same for the riding level l2
  const int* tlist;      // gathered levels: target cells grouped by class
  const int* toff;       // gathered levels: offsets of the classes in tlist [9]
  const char* ghi;       // gathered levels: the window's rows (hi, lo), JP per row
  const char* glo;
  float scale, scale2;   // exact powers of two (shared offset matrices)
  int l, BX, BY, BZ, ntx, nty, first_block, Hx, Hy, Hz;
  int l2;
  int gather, zero_row;
};
constexpr int kTcMaxLevels = 10;
struct TcParams {
  TcLevel lev[kTcMaxLevels];
  int nlev, nj, jchunks, ksteps_last;
  int nc, npt, ncls;   // columns per block, rows per offset matrix, stacked classes
  int nstages, stage_bytes;
  int accumulate;      // add into the local expansions (else store)
  long long wait_cycles;  // limit of the pipeline's mbarrier waits
  int* err;
  // F16X3: the table norm (tc_norm at table level tlev_fixed, or at the CTA's
  // level when 0) and m! of the local coefficients
  const Geom* geom;
  int kernel, tlev_fixed;
  const float* fact_f;
};

// F16X3: where the scale 2^e_box of the source box feeding TMEM lane `row`
// is found, packed in one register (the drain has none to spare): the row's
// parent (x, y, z) in its level's cell grid (hx, hy, hz) gives
// base = (z hy + y) hx + x (< 2^21 for levels <= 8), bits 21..26 flag the
// neighbours that exist (x-1, x+1, y-1, y+1, z-1, z+1), bit 27 the riding
// level's rows and bit 28 a loaded row inside its grid (0: no source).
__device__ __forceinline__ int row_scale_setup(const TcLevel& LV, int row, int N1, int NR, int X0,
                                               int Y0, int Z0, int BX, int BY, int H2) {
  if (row >= NR) return 0;
  int x, y, z, hx, hy, hz, ride = 0;
  if (row < N1) {
    x = X0 + row % BX;
    y = Y0 + (row / BX) % BY;
    z = Z0 + row / (BX * BY);
    hx = LV.Hx;
    hy = LV.Hy;
    hz = LV.Hz;
  } else {
    const int n2 = row - N1;
    x = n2 % H2;
    y = (n2 / H2) % H2;
    z = n2 / (H2 * H2);
    hx = hy = hz = H2;
    ride = 1;
  }
  if (x >= hx || y >= hy || z >= hz) return 0;  // a target outside the grid: not stored
  const int mask = (x > 0) | ((x + 1 < hx) << 1) | ((y > 0) << 2) | ((y + 1 < hy) << 3) |
                   ((z > 0) << 4) | ((z + 1 < hz) << 5) | (ride << 6) | (1 << 7);
  return ((z * hy + y) * hx + x) | (mask << 21);
}

// 2^e_box of the source (child sg of the parent shifted by (dx, dy, dz)); 0
// for a source outside the grid, whose TMA rows are zero
__device__ __forceinline__ float row_scale(const TcLevel& LV, int H2, int rb, int sg, int dx,
                                           int dy, int dz) {
  const int mask = rb >> 21;
  if (!(mask & 128)) return 0.f;
  const bool ok = (dx >= 0 || (mask & 1)) && (dx <= 0 || (mask & 2)) &&
                  (dy >= 0 || (mask & 4)) && (dy <= 0 || (mask & 8)) &&
                  (dz >= 0 || (mask & 16)) && (dz <= 0 || (mask & 32));
  if (!ok) return 0.f;
  const bool ride = mask & 64;
  const int hx = ride ? H2 : LV.Hx, hy = ride ? H2 : LV.Hy, hz = ride ? H2 : LV.Hz;
  const float* bs = ride ? LV.bscale2 : LV.bscale;
  return bs[(rb & 0x1fffff) + ((sg * hz + dz) * hy + dy) * hx + dx];
}

// pipeline wait: the default bounded wait, or (SHORTW, the instantiation that
// tests run with a shortened limit) the polling wait of mbar_wait_short
template <bool SHORTW>
__device__ __forceinline__ bool pwait(uint64_t* bar, uint32_t parity, int* err, long long lim) {
  return SHORTW ? tc::mbar_wait_short(bar, parity, err, lim) : tc::mbar_wait(bar, parity, err);
}

template <typename F, int NPASS, bool SHORTW, int NCOL>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_m2l_tc(const __grid_constant__ TcParams prm) {
  using C = Cfg<NPASS>;
  int li = 0;
  while (li + 1 < prm.nlev && (int)blockIdx.x >= prm.lev[li + 1].first_block) ++li;
  const TcLevel& LV = prm.lev[li];
  const int l = LV.l, nj = prm.nj, jchunks = prm.jchunks;
  const int nc = prm.nc, npt = prm.npt, ncls = prm.ncls;
  const int ntot = nc * ncls;  // MMA N
  const int ns = prm.nstages, sbytes = prm.stage_bytes;
  const int btile = ntot * C::kRowBytes;  // offset-matrix bytes of one stage half
  const int BX = LV.BX, BY = LV.BY, BZ = LV.BZ, ntx = LV.ntx, nty = LV.nty;
  int* __restrict__ err = prm.err;
  const long long wlim = prm.wait_cycles;
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + ns * sbytes);
  uint64_t* empty = full + kMaxStages;
  uint64_t* accf = empty + kMaxStages;  // [kNBuf] accumulator filled (MMA commit)
  uint64_t* acce = accf + kNBuf;        // [kNBuf] accumulator drained (warp arrivals)
  uint64_t* drainb = acce + kNBuf;      // all MMAs of this CTA finished
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drainb + 1);
  int* bad = reinterpret_cast<int*>(tslot + 1);  // a draining warp gave up

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lb = (int)blockIdx.x - LV.first_block;
  const int ngrp = 8 / ncls;
  int pi0 = (lb % ngrp) * ncls;  // classes pi0 .. pi0 + ncls - 1
  const int tile = LV.gather ? 0 : lb / ngrp;
  int gstart = 0, grows = 0;  // gathered levels: this CTA's entries of tlist
  if (LV.gather) {  // (ncls == 1) block lb: entries 128 (lb / 8).. of class lb % 8
    pi0 = lb & 7;
    const int n = LV.toff[pi0 + 1] - LV.toff[pi0], k0 = (lb >> 3) * kBM;
    if (k0 >= n) return;  // a surplus CTA: block-uniform, before any barrier or TMEM
    gstart = LV.toff[pi0] + k0;
    grows = min(kBM, n - k0);
  }
  const int cb = blockIdx.y;  // column block
  const int tx = tile % ntx, ty = (tile / ntx) % nty, tz = tile / (ntx * nty);
  const int X0 = tx * BX, Y0 = ty * BY, Z0 = tz * BZ;
  const int l2 = LV.l2, H2 = l2 ? 1 << (l2 - 1) : 0;
  const int N1 = BX * BY * BZ;      // source rows of the primary tile
  const int NR = N1 + H2 * H2 * H2;  // rows the TMA boxes fill (<= 128)

  if (LV.map && !LV.gather) {  // a window's tile whose target cells hold no box: nothing to do
    int any = 0;
    for (int e = threadIdx.x; e < N1 * ncls; e += blockDim.x) {
      const int n = e % N1, u = e / N1;
      const int x = X0 + n % BX, y = Y0 + (n / BX) % BY, z = Z0 + n / (BX * BY);
      if (x < LV.Hx && y < LV.Hy && z < LV.Hz)
        any |= LV.map[(((size_t)(pi0 + u) * LV.Hz + z) * LV.Hy + y) * LV.Hx + x] >= 0;
    }
    if (!__syncthreads_or(any)) return;  // block-uniform, before any barrier or TMEM
  }

  if (threadIdx.x == 0) {
    for (int s = 0; s < ns; ++s) {
      // gathered levels: lane 0's arm plus the 32 lanes' copy arrivals
      tc::mbar_init(&full[s], LV.gather ? 33 : 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int bf = 0; bf < kNBuf; ++bf) {
      tc::mbar_init(&accf[bf], 1);
      tc::mbar_init(&acce[bf], kEpiWarps);
    }
    tc::mbar_init(drainb, 1);
    *bad = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tslot, kTmemCols);

  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;

  if (warp == kEpiWarps && LV.gather) {
    // ---------------- producer, gathered rows ----------------
    // The 32 lanes copy the 128 source rows of each stage with cp.async, 16
    // bytes at a time, into the 128-byte-swizzled layout (lane i: 16-byte
    // column i % 8 of rows i / 8 + 4k) and arrive on the stage barrier when
    // their copies land; lane 0 also waits for free stages and loads the
    // offset matrices by TMA.
    const uint32_t stage_tx = (uint32_t)C::kHalves * (uint32_t)btile;  // the TMA part
    const size_t pitch = (size_t)jchunks * C::kRowBytes;              // bytes per window row
    int* rowix = reinterpret_cast<int*>(sm + ns * sbytes + 256);      // [kBM] source rows
    const int Hx = LV.Hx, Hy = LV.Hy, Hz = LV.Hz;
    const int q16 = lane & 7, r0 = lane >> 3;
    int cx[4], cy[4], cz[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = 4 * lane + j;
      cx[j] = cy[j] = cz[j] = -4;  // no target: every source outside the window
      if (n < grows) {
        const int cell = LV.tlist[gstart + n];
        cx[j] = cell % Hx;
        cy[j] = (cell / Hx) % Hy;
        cz[j] = cell / (Hx * Hy);
      }
    }
    int s = 0, kk = 0;
    uint32_t ph = 0;
    unsigned char* st = sm;
    int last_par[kMaxStages];  // (lane 0) parity of the last round armed in a stage
    for (int q = 0; q < kMaxStages; ++q) last_par[q] = -1;
    bool ok = true;
    for (int c = 0; c < 216 && ok; ++c) {
      const Combo k = combo(c);
      if (!any_far(k, pi0, 1)) continue;
      __syncwarp();  // the previous combination's rows have been read
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int x = cx[j] + k.dx, y = cy[j] + k.dy, z = cz[j] + k.dz;
        rowix[4 * lane + j] = (x >= 0 && x < Hx && y >= 0 && y < Hy && z >= 0 && z < Hz)
                                  ? ((k.sg * Hz + z) * Hy + y) * Hx + x
                                  : LV.zero_row;
      }
      __syncwarp();
      bool f;
      const int hidx = offset_of(k, pi0, &f) * npt + cb * nc;
      for (int ch = 0; ch < jchunks; ++ch, ++kk) {
        int go = 1;
        if (lane == 0) {
          if (kk >= ns && !pwait<SHORTW>(&empty[s], ph ^ 1u, err, wlim)) {
            go = 0;
          } else {
            tc::mbar_expect_tx(&full[s], stage_tx);
            last_par[s] = (int)ph;
          }
        }
        if (!__shfl_sync(0xffffffffu, go, 0)) {  // the stage is free before any copy
          ok = false;
          break;
        }
#pragma unroll
        for (int hf = 0; hf < C::kHalves; ++hf) {
          unsigned char* sh = st + hf * (C::kTileS + btile);
          const char* g = (hf ? LV.glo : LV.ghi) + (size_t)ch * C::kRowBytes + q16 * 16;
#pragma unroll 8
          for (int i = 0; i < kBM / 4; ++i) {
            const int rr = r0 + 4 * i;
            tc::cp_async16(sh + rr * C::kRowBytes + ((q16 ^ (rr & 7)) << 4),
                           g + (size_t)rowix[rr] * pitch);
          }
          if (lane == 0)
            tc::tma_load_2d(sh + C::kTileS, hf ? &LV.Hlo : &LV.H, &full[s], ch * (C::kRowBytes /
                            (int)sizeof(typename F::T)), hidx);
        }
        tc::cp_async_arrive(&full[s]);
        if (++s == ns) {
          s = 0;
          ph ^= 1u;
          st = sm;
        } else {
          st += sbytes;
        }
      }
    }
    tc::cp_async_wait_all();  // every copy of this warp has landed before it leaves
    if (!ok && lane == 0) {  // TMA copies still in flight before the CTA leaves
      for (int q = 0; q < ns; ++q)
        if (last_par[q] >= 0) {
          const long long t0 = clock64();
          while (!tc::mbar_try_wait(&full[q], (uint32_t)last_par[q]) &&
                 clock64() - t0 < tc::kWaitCycles) {
          }
        }
    }
  } else if (warp == kEpiWarps && lane == 0) {
    // ---------------- TMA producer ----------------
    // stage s and the parity ph of its current round advance together (no
    // division in the loop); a stage is refilled once its previous round's
    // MMAs have committed
    const uint32_t bytesS = (uint32_t)NR * C::kRowBytes;
    const uint32_t stage_tx = (uint32_t)C::kHalves * (bytesS + (uint32_t)btile);
    constexpr int kElems = C::kRowBytes / (int)sizeof(typename F::T);
    int s = 0, kk = 0;
    uint32_t ph = 0;
    unsigned char* st = sm;
    int last_par[kMaxStages];  // parity of the last round issued into a stage (-1: none)
    for (int q = 0; q < kMaxStages; ++q) last_par[q] = -1;
    bool ok = true;
    for (int c = 0; c < 216 && ok; ++c) {
      const Combo k = combo(c);
      if (!any_far(k, pi0, ncls)) continue;
      int hidx[8];
      for (int u = 0; u < ncls; ++u) {
        bool f;
        hidx[u] = offset_of(k, pi0 + u, &f) * npt + cb * nc;
      }
      for (int ch = 0; ch < jchunks; ++ch, ++kk) {
        if (kk >= ns && !pwait<SHORTW>(&empty[s], ph ^ 1u, err, wlim)) {
          ok = false;
          break;
        }
        tc::mbar_expect_tx(&full[s], stage_tx);
        last_par[s] = (int)ph;
        const int kc = ch * kElems;  // element offset of this K chunk
#pragma unroll
        for (int hf = 0; hf < C::kHalves; ++hf) {
          unsigned char* sh = st + hf * (C::kTileS + btile);
          tc::tma_load_5d(sh, hf ? &LV.Slo : &LV.S, &full[s], kc, X0 + k.dx, Y0 + k.dy,
                          Z0 + k.dz, k.sg);
          if (l2)  // N1 is a multiple of 8 rows: the second box starts on a swizzle atom
            tc::tma_load_5d(sh + N1 * C::kRowBytes, hf ? &LV.S2lo : &LV.S2, &full[s], kc, k.dx,
                            k.dy, k.dz, k.sg);
          for (int u = 0; u < ncls; ++u)
            tc::tma_load_2d(sh + C::kTileS + u * nc * C::kRowBytes, hf ? &LV.Hlo : &LV.H,
                            &full[s], kc, hidx[u]);
        }
        if (++s == ns) {
          s = 0;
          ph ^= 1u;
          st = sm;
        } else {
          st += sbytes;
        }
      }
    }
    if (!ok) {  // drain copies still in flight before the CTA leaves
      for (int q = 0; q < ns; ++q)
        if (last_par[q] >= 0) {
          const long long t0 = clock64();
          while (!tc::mbar_try_wait(&full[q], (uint32_t)last_par[q]) &&
                 clock64() - t0 < tc::kWaitCycles) {
          }
        }
    }
  } else if (warp == kEpiWarps + 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    // everything between two MMAs is kept to a few adds: descriptors advance
    // by the stage size, the stage index and parity by increments
    const uint32_t id = tc::idesc(F::kIdesc, kBM, ntot);
    const uint64_t d0 = C::desc(tc::smem_u32(sm));
    const uint64_t ob = (uint64_t)(C::kTileS >> 4);
    const uint64_t oalo = (uint64_t)((C::kTileS + btile) >> 4);
    const uint64_t oblo = (uint64_t)((2 * C::kTileS + btile) >> 4);
    const uint64_t dstep = (uint64_t)(sbytes >> 4);
    const int kl = prm.ksteps_last;
    const bool gath = LV.gather != 0;
    int s = 0;
    uint32_t ph = 0;
    uint64_t da = d0;
    int g = 0;  // offsets issued: buffer g & 1, its (g >> 1)-th use
    bool ok = true;
    for (int c = 0; c < 216 && ok; ++c) {
      const Combo k = combo(c);
      if (!any_far(k, pi0, ncls)) continue;
      const int bf = g & 1;
      if (g >= kNBuf && !pwait<SHORTW>(&acce[bf], ((g >> 1) - 1) & 1, err, wlim)) {
        ok = false;  // the buffer's previous offset has not been drained
        break;
      }
      tc::fence_after();
      const uint32_t dacc = tmem + (uint32_t)(bf * kMaxN);
      for (int ch = 0; ch < jchunks; ++ch) {
        if (!pwait<SHORTW>(&full[s], ph, err, wlim)) {
          ok = false;
          break;
        }
        tc::fence_after();
        if (gath) tc::fence_proxy_async();  // the copies went through the generic proxy
        const int nk = ch == jchunks - 1 ? kl : C::kKSteps;
#pragma unroll
        for (int ks = 0; ks < C::kKSteps; ++ks) {
          if (ks < nk) {
            // one MMA consumes 32 bytes of K (8 tf32 or 16 bf16) inside the swizzle atom
            const uint64_t a = da + (uint64_t)(ks * 2);
            const uint32_t acc = (ch | ks) != 0;
            if (F::kF16) {
              tc::mma_f16(dacc, a, a + ob, id, acc);
              if (NPASS == 3) {
                tc::mma_f16(dacc, a, a + oblo, id, 1);
                tc::mma_f16(dacc, a + oalo, a + ob, id, 1);
              }
            } else {
              tc::mma_tf32(dacc, a, a + ob, id, acc);
              if (NPASS == 3) {
                tc::mma_tf32(dacc, a, a + oblo, id, 1);
                tc::mma_tf32(dacc, a + oalo, a + ob, id, 1);
              }
            }
          }
        }
        tc::mma_commit(&empty[s]);
        if (++s == ns) {
          s = 0;
          ph ^= 1u;
          da = d0;
        } else {
          da += dstep;
        }
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
    const int quad = warp & 3;
    const int cw = (ntot / (kEpiWarps / 4) + 7) / 8 * 8;  // columns of this warp's group
    const int c0 = (warp >> 2) * cw;
    float sum[NCOL];
#pragma unroll
    for (int j = 0; j < NCOL; ++j) sum[j] = 0.f;
    bool ok = true;
    int g = 0;
    const int row = quad * 32 + lane;  // this thread's TMEM lane
    const int rb = F::kScaled ? row_scale_setup(LV, row, N1, NR, X0, Y0, Z0, BX, BY, H2) : 0;
    for (int c = 0; c < 216; ++c) {
      const Combo kc = combo(c);
      if (!any_far(kc, pi0, ncls)) continue;
      const int bf = g & 1;
      // F16X3: the power of two the row's source multipole was divided by
      // (read before the wait, off the critical path)
      const float rs =
          F::kScaled ? row_scale(LV, H2, rb, kc.sg, kc.dx, kc.dy, kc.dz) : 1.f;
      if (!pwait<SHORTW>(&accf[bf], (g >> 1) & 1, err, wlim)) {
        ok = false;
        break;
      }
      tc::fence_after();
      const uint32_t base =
          tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(bf * kMaxN + c0);
      // pairs of 8-column groups: loaded, then summed (16 registers in flight)
#pragma unroll
      for (int gp = 0; gp < NCOL / 16; ++gp) {
        uint32_t r0[8], r1[8];
        const bool v0 = 16 * gp < cw && c0 + 16 * gp < ntot;
        const bool v1 = 16 * gp + 8 < cw && c0 + 16 * gp + 8 < ntot;
        if (v0) tc::tmem_ld8_nowait(base + (uint32_t)(16 * gp), r0);
        if (v1) tc::tmem_ld8_nowait(base + (uint32_t)(16 * gp + 8), r1);
        if (v0 || v1) tc::tmem_wait();
        if (v0) {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            sum[16 * gp + j] = F::kScaled ? fmaf(__uint_as_float(r0[j]), rs, sum[16 * gp + j])
                                          : sum[16 * gp + j] + __uint_as_float(r0[j]);
        }
        if (v1) {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            sum[16 * gp + 8 + j] =
                F::kScaled ? fmaf(__uint_as_float(r1[j]), rs, sum[16 * gp + 8 + j])
                           : sum[16 * gp + 8 + j] + __uint_as_float(r1[j]);
        }
      }
      tc::fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[bf]);
      ++g;
    }
    // every draining warp passes both barriers below, whatever its status, so
    // that none waits for a warp that left; the decision to write is taken
    // from shared memory after the first barrier, the same for all
    if (!ok || (*(volatile int*)err & 2)) atomicOr(bad, 1);
    drain_sync();
    const bool good = *(volatile int*)bad == 0;
    // every MMA has finished and every TMA copy has been consumed: the stage
    // memory is free for the staging of the sums, [row][column] with an odd
    // pitch (the 32 lanes of a warp write 32 rows of one column)
    float* stg = reinterpret_cast<float*>(sm);
    const int pitch = ntot + 1;
    if (good) {
#pragma unroll
      for (int j = 0; j < NCOL; ++j)
        if (j < cw && c0 + j < ntot) stg[row * pitch + c0 + j] = sum[j];
    }
    drain_sync();
    if (good) {
      const int nv = min(nc, nj - cb * nc);  // valid columns of this block
      // F16X3: the table norm of the offset matrices this level used
      const float tn = F::kScaled ? (float)tc_norm(prm.kernel, prm.geom->size,
                                                   prm.tlev_fixed ? prm.tlev_fixed : l)
                                  : 1.f;
      const int nl = 1 << l, Hx = LV.Hx, Hy = LV.Hy, Hz = LV.Hz;
      const int* __restrict__ map = LV.map;
      const int tot = NR * ncls * nv;
      for (int e = threadIdx.x; e < tot; e += kEpiWarps * 32) {
        const int i = e % nv, rc = e / nv;
        const int u = rc % ncls, n = rc / ncls;
        const int pi = pi0 + u;
        const int px = pi & 1, py = (pi >> 1) & 1, pz = (pi >> 2) & 1;
        float v = stg[n * pitch + u * nc + i];
        if (F::kScaled) v *= prm.fact_f[cb * nc + i] * tn;  // S_i and the table norm
        double* dst = nullptr;
        double scale = 1.0;
        if (LV.gather) {  // row n: entry gstart + n of the class list
          if (n < grows) {
            const int64_t t = (int64_t)map[(size_t)pi * Hz * Hy * Hx + LV.tlist[gstart + n]];
            if (t >= 0) dst = LV.lc + t * nj + cb * nc + i;
            scale = LV.scale;
          }
        } else if (n < N1) {
          const int x = X0 + n % BX, y = Y0 + (n / BX) % BY, z = Z0 + n / (BX * BY);
          if (x < Hx && y < Hy && z < Hz) {
            const int64_t t =
                map ? (int64_t)map[(((size_t)pi * Hz + z) * Hy + y) * Hx + x]
                    : ((int64_t)(2 * z + pz) * nl + (2 * y + py)) * nl + (2 * x + px);
            if (t >= 0) dst = LV.lc + t * nj + cb * nc + i;
            scale = LV.scale;
          }
        } else {  // the riding level's targets
          const int n2 = n - N1, nl2 = 2 * H2;
          const int x = n2 % H2, y = (n2 / H2) % H2, z = n2 / (H2 * H2);
          const int64_t t = ((int64_t)(2 * z + pz) * nl2 + (2 * y + py)) * nl2 + (2 * x + px);
          dst = LV.lc2 + t * nj + cb * nc + i;
          scale = LV.scale2;
        }
        if (dst) {
          const double val = (double)(v * (float)scale);
          if (prm.accumulate) *dst += val;
          else *dst = val;
        }
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
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

// Target tile of a parent grid Hx x Hy x Hz: up to 8 x 4 x 4 = 128 parents,
// x fastest.
void tile_shape(int Hx, int Hy, int Hz, TcLevel* v) {
  v->BX = std::min(8, Hx);
  v->BZ = std::min(4, Hz);
  v->BY = std::min(Hy, kBM / (v->BX * v->BZ));
  v->ntx = (Hx + v->BX - 1) / v->BX;
  v->nty = (Hy + v->BY - 1) / v->BY;
}

// the launch parameters that do not depend on the level
template <typename F, int NPASS>
bool common_params(const fmm_plan_s* P, const Workspace& ws, TcParams* prm) {
  using C = Cfg<NPASS>;
  const TcShape sh = tc_shape(P->pd.nj, P->desc.precision);
  std::memset(prm, 0, sizeof(*prm));
  prm->nj = P->pd.nj;
  const int row = C::kRowBytes / (int)sizeof(typename F::T);  // elements per K chunk
  if (sh.row_bytes != C::kRowBytes || ws.tc_jp != sh.jp || ws.tc_mp != sh.npt) return false;
  prm->jchunks = ws.tc_jp / row;
  const int kstep = 32 / (int)sizeof(typename F::T);  // elements of K per MMA
  const int ksteps = (P->pd.nj + kstep - 1) / kstep;
  prm->ksteps_last = ksteps - (prm->jchunks - 1) * C::kKSteps;
  prm->nc = sh.nc;
  prm->npt = sh.npt;
  prm->ncls = sh.ncls;
  prm->stage_bytes = C::stage_bytes(sh.nc * sh.ncls);
  prm->nstages = std::min(kMaxStages, (kSmemCap - 1024 - 256 - kBM * (int)sizeof(int)) / prm->stage_bytes);
  prm->wait_cycles = P->tc_wait_cycles > 0 ? P->tc_wait_cycles : tc::kWaitCycles;
  prm->err = &ws.geom->flag;
  // the staging of the sums reuses the stages
  if (kBM * (sh.nc * sh.ncls + 1) * (int)sizeof(float) > prm->nstages * prm->stage_bytes)
    return false;
  return prm->nstages >= 2 && prm->ksteps_last >= 1 && prm->ksteps_last <= C::kKSteps;
}

template <typename F, int NPASS>
size_t smem_bytes(const TcParams& prm) {
  return 1024 + (size_t)prm.nstages * prm.stage_bytes + 256 + kBM * sizeof(int);
}

// offset matrices A_h (hi and lo) of a uniform tree from the derivative tables
template <typename F, int NPASS>
void build_tables(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st, int tlev) {
  using T = typename F::T;
  const PlanDev& pd = P->pd;
  T* thi0 = static_cast<T*>(ws.tc_tmat[0]);
  T* tlo = NPASS == 3 ? static_cast<T*>(ws.tc_tmat[1]) : nullptr;
  const size_t sm = std::max(2 * sizeof(T) * pd.nh, sizeof(double) * pd.nj);
  if (sm > 48 * 1024)
    cudaFuncSetAttribute(k_build_tmat<3, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_build_tmat<3, F><<<dim3(343, tlev), 256, sm, st>>>(pd, ws.geom, ws.htab, ws.tc_mp, ws.tc_jp,
                                                       thi0, tlo);
}

// tensor maps of the offset matrices of table level ti
template <typename F, int NPASS>
bool offset_maps(const Workspace& ws, int ti, const TcParams& prm, TcLevel* v) {
  using C = Cfg<NPASS>;
  using T = typename F::T;
  const size_t esz = sizeof(T);
  const CUtensorMapDataType dt = F::kMapType;
  const int JP = ws.tc_jp, NPT = ws.tc_mp, row = C::kRowBytes / (int)esz;
  const size_t per = (size_t)343 * NPT * JP;
  cuuint64_t dA[2] = {(cuuint64_t)JP, (cuuint64_t)343 * NPT};
  cuuint64_t sA[1] = {(cuuint64_t)JP * esz};
  cuuint32_t bA[2] = {(cuuint32_t)row, (cuuint32_t)prm.nc};
  T* thi = static_cast<T*>(ws.tc_tmat[0]) + (size_t)ti * per;
  if (!make_map(&v->H, thi, 2, dA, sA, bA, dt, C::kRowBytes)) return false;
  v->Hlo = v->H;
  if (NPASS == 3) {
    T* tlo = static_cast<T*>(ws.tc_tmat[1]) + (size_t)ti * per;
    if (!make_map(&v->Hlo, tlo, 2, dA, sA, bA, dt, C::kRowBytes)) return false;
  }
  return true;
}

// tensor map of parity-split multipoles Bpar[8][Hz][Hy][Hx][JP], box of
// (bx, by, bz) parents
template <typename F, int NPASS>
bool source_map(CUtensorMap* m, void* base, int JP, int Hx, int Hy, int Hz, int bx, int by,
                int bz) {
  using C = Cfg<NPASS>;
  const size_t esz = sizeof(typename F::T);
  const CUtensorMapDataType dt = F::kMapType;
  const int row = C::kRowBytes / (int)esz;
  cuuint64_t dB[5] = {(cuuint64_t)JP, (cuuint64_t)Hx, (cuuint64_t)Hy, (cuuint64_t)Hz, 8};
  cuuint64_t sB[4] = {(cuuint64_t)JP * esz, (cuuint64_t)JP * esz * Hx,
                      (cuuint64_t)JP * esz * Hx * Hy, (cuuint64_t)JP * esz * Hx * Hy * Hz};
  cuuint32_t bB[5] = {(cuuint32_t)row, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz, 1};
  return make_map(m, base, 5, dB, sB, bB, dt, C::kRowBytes);
}

template <typename F, int NPASS, bool SHORTW, int NCOL>
void launch_variant(const TcParams& prm, dim3 grid, size_t sm, cudaStream_t st) {
  cudaFuncSetAttribute(k_m2l_tc<F, NPASS, SHORTW, NCOL>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_m2l_tc<F, NPASS, SHORTW, NCOL><<<grid, kTcThreads, sm, st>>>(prm);
}

template <typename F, int NPASS>
cudaError_t launch_contraction(const fmm_plan_s* P, const TcParams& prm, int nb, cudaStream_t st,
                               bool timed) {
  const size_t sm = smem_bytes<F, NPASS>(prm);
  const TcShape sh = tc_shape(P->pd.nj, P->desc.precision);
  const dim3 grid(nb, sh.nchunk);
  // a drain warp's columns: cw = N / 4 rounded up to 8
  const bool small = ((prm.nc * prm.ncls) / (kEpiWarps / 4) + 7) / 8 * 8 <= kColsSmall;
  // per call: the attribute belongs to the current device's context
  if (timed) mark_contraction(P, 0, st);
  if (prm.wait_cycles < tc::kWaitCycles) {  // a test's shortened waits
    if (small) launch_variant<F, NPASS, true, kColsSmall>(prm, grid, sm, st);
    else launch_variant<F, NPASS, true, kColsLarge>(prm, grid, sm, st);
  } else {
    if (small) launch_variant<F, NPASS, false, kColsSmall>(prm, grid, sm, st);
    else launch_variant<F, NPASS, false, kColsLarge>(prm, grid, sm, st);
  }
  if (timed) mark_contraction(P, 1, st);
  return cudaGetLastError();
}

template <typename F, int NPASS>
cudaError_t run_all_levels(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st,
                           bool tables_ready) {
  const PlanDev& pd = P->pd;
  const int L = P->desc.levels;
  const int nj = pd.nj, JP = ws.tc_jp;
  const bool shared_t = kernel_homogeneous(pd.kernel);  // G(s h) = s^deg G(h)
  const int tlev = shared_t ? 1 : (L - 1);
  using T = typename F::T;
  T* bhi0 = static_cast<T*>(ws.tc_bpar[0]);
  T* blo = NPASS == 3 ? static_cast<T*>(ws.tc_bpar[1]) : nullptr;
  LevOff lo;
  for (int l = 0; l <= FMM_MAX_LEVELS; ++l) lo.o[l] = l <= L + 1 ? ws.lev_off[l] : 0;
  if (F::kScaled)
    k_pack_beta_scaled<F><<<dim3(152 * 4, L - 1), 256, 0, st>>>(ws.mp, lo, nj, JP, pd.fact_f,
                                                                bhi0, blo, ws.tc_bscale);
  else
    k_pack_beta<F><<<dim3(152 * 4, L - 1), 256, 0, st>>>(ws.mp, lo, nj, JP, bhi0, blo);
  if (!tables_ready) build_tables<F, NPASS>(P, ws, st, tlev);
  TcParams prm;
  if (!common_params<F, NPASS>(P, ws, &prm)) return cudaErrorInvalidValue;
  prm.accumulate = 0;  // every coefficient of levels 2..L is written exactly once
  prm.geom = ws.geom;
  prm.kernel = pd.kernel;
  prm.tlev_fixed = shared_t ? 2 : 0;  // shared tables are level 2's
  prm.fact_f = pd.fact_f;
  const int ngrp = 8 / prm.ncls;
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
    nb += v.ntx * v.nty * ntz * ngrp;
    v.lc = ws.lc + ws.lev_off[l] * nj;
    v.map = nullptr;
    v.bscale = F::kScaled ? ws.tc_bscale + ws.lev_off[l] : nullptr;
    v.bscale2 = nullptr;
    v.Hx = v.Hy = v.Hz = H;
    v.scale = 1.0f;
    if (shared_t) {  // Ht_l = Ht_2 * (s_2/s_l)^{-deg}: deg -1 (Laplace), +1 (biharmonic)
      const int k = l - 2;
      v.scale = pd.kernel == FMM_KERNEL_LAPLACE ? std::ldexp(1.0f, k) : std::ldexp(1.0f, -k);
    }
    if (!offset_maps<F, NPASS>(ws, shared_t ? 0 : l - 2, prm, &v)) return cudaErrorInvalidValue;
    if (!source_map<F, NPASS>(&v.S, bhi0 + ws.lev_off[l] * JP, JP, H, H, H, v.BX, v.BY, v.BZ))
      return cudaErrorInvalidValue;
    v.Slo = v.S;
    if (NPASS == 3 &&
        !source_map<F, NPASS>(&v.Slo, blo + ws.lev_off[l] * JP, JP, H, H, H, v.BX, v.BY, v.BZ))
      return cudaErrorInvalidValue;
    if (l == 3 && lmin == 3) {  // level 2: 2 x 2 x 2 parents after level 3's 64
      v.l2 = 2;
      v.lc2 = ws.lc + ws.lev_off[2] * nj;
      v.bscale2 = F::kScaled ? ws.tc_bscale + ws.lev_off[2] : nullptr;
      v.scale2 = 1.0f;
      if (!source_map<F, NPASS>(&v.S2, bhi0 + ws.lev_off[2] * JP, JP, 2, 2, 2, 2, 2, 2))
        return cudaErrorInvalidValue;
      v.S2lo = v.S2;
      if (NPASS == 3 &&
          !source_map<F, NPASS>(&v.S2lo, blo + ws.lev_off[2] * JP, JP, 2, 2, 2, 2, 2, 2))
        return cudaErrorInvalidValue;
    }
  }
  return launch_contraction<F, NPASS>(P, prm, nb, st, true);
}

// ---- adaptive trees: every level packed into a dense window ----------------
// (the windows come from the tree's per-level coordinate bounds, read with its
// level offsets)

// the level's boxes into Bpar[sigma][Tz][Ty][Tx][JP] (hi and lo) of a window
// with parent origin W and size H, and map[sigma][Tz][Ty][Tx] = box; one warp
// per box (the box's cell found once, the lanes over its coefficients)
template <typename F>
__global__ void __launch_bounds__(256) k_apack(ATree t, int l, const double* __restrict__ mp,
                                               int nj, int JP, int W0x, int W0y, int W0z, int Hx,
                                               int Hy, int Hz, typename F::T* __restrict__ bhi,
                                               typename F::T* __restrict__ blo,
                                               int* __restrict__ map) {
  const int b0 = t.loff[l], nbl = t.loff[l + 1] - b0;
  const int lane = threadIdx.x & 31;
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  for (int bi = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); bi < nbl; bi += nw) {
    const int b = b0 + bi;
    int c[3];
    demorton3(t.key[b], l, c);
    const int sg = (c[0] & 1) | ((c[1] & 1) << 1) | ((c[2] & 1) << 2);
    const size_t cell =
        (((size_t)sg * Hz + ((c[2] >> 1) - W0z)) * Hy + ((c[1] >> 1) - W0y)) * Hx + ((c[0] >> 1) - W0x);
    const double* src = mp + (size_t)b * nj;
    for (int q = lane; q < JP; q += 32) {
      const float v = q < nj ? (float)src[q] : 0.f;
      typename F::T hi, lo;
      F::split(v, hi, lo);
      bhi[cell * JP + q] = hi;
      if (blo) blo[cell * JP + q] = lo;
    }
    if (lane == 0) map[cell] = t.t1[b] > t.t0[b] ? b : -1;  // only boxes with targets get locals
  }
}

// The target cells of level l (boxes holding targets, parent cell in the
// window with parent origin W and size H) grouped by class: toff[u] is where
// class u starts in tlist, toff[8] the total; inside a class the cells keep
// the boxes' Morton order (one block of 1024 threads per level: class counts,
// then positions by warp ballots and a prefix over the warps of each chunk).
__global__ void __launch_bounds__(1024) k_alist(ATree t, int l, int W0x, int W0y, int W0z,
                                                int Hx, int Hy, int* __restrict__ tlist,
                                                int* __restrict__ toff) {
  __shared__ int wcnt[32][8];
  __shared__ int base[8];
  const int b0 = t.loff[l], n = t.loff[l + 1] - b0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x < 8) base[threadIdx.x] = 0;
  __syncthreads();
  auto classify = [&](int i, int* cell) {
    if (i >= n || t.t1[b0 + i] == t.t0[b0 + i]) return -1;
    int c[3];
    demorton3(t.key[b0 + i], l, c);
    *cell = (((c[2] >> 1) - W0z) * Hy + ((c[1] >> 1) - W0y)) * Hx + ((c[0] >> 1) - W0x);
    return (c[0] & 1) | ((c[1] & 1) << 1) | ((c[2] & 1) << 2);
  };
  for (int i0 = 0; i0 < n; i0 += 1024) {  // class counts
    int cell;
    const int cls = classify(i0 + (int)threadIdx.x, &cell);
    for (int u = 0; u < 8; ++u) {
      const unsigned m = __ballot_sync(0xffffffffu, cls == u);
      if (lane == 0 && m) atomicAdd(&base[u], __popc(m));
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int u = 0; u < 8; ++u) {
      const int c = base[u];
      base[u] = acc;
      toff[u] = acc;
      acc += c;
    }
    toff[8] = acc;
  }
  __syncthreads();
  for (int i0 = 0; i0 < n; i0 += 1024) {  // positions
    int cell = 0;
    const int cls = classify(i0 + (int)threadIdx.x, &cell);
    unsigned mine = 0;
    for (int u = 0; u < 8; ++u) {
      const unsigned m = __ballot_sync(0xffffffffu, cls == u);
      if (lane == 0) wcnt[warp][u] = __popc(m);
      if (cls == u) mine = m;
    }
    __syncthreads();
    if (cls >= 0) {
      int pos = base[cls] + __popc(mine & ((1u << lane) - 1u));
      for (int w = 0; w < warp; ++w) pos += wcnt[w][cls];
      tlist[pos] = cell;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
      int add = 0;
      for (int w = 0; w < 32; ++w) add += wcnt[w][threadIdx.x];
      base[threadIdx.x] += add;
    }
    __syncthreads();
  }
}

template <typename F, int NPASS>
cudaError_t run_adaptive(const fmm_plan_s* P, const Workspace& ws, const ATree& t,
                         cudaStream_t st, int* nl, unsigned* done) {
  using T = typename F::T;
  const PlanDev& pd = P->pd;
  const int nj = pd.nj, JP = ws.tc_jp;
  const bool shared_t = kernel_homogeneous(pd.kernel);  // G(s h) = s^deg G(h)
  const int tlev = shared_t ? 1 : (t.maxlev - 1);
  const size_t esz = sizeof(T);
  // coordinate bounds of every level, read with the tree's level offsets
  const int* bnd = P->abnd;
  build_tables<F, NPASS>(P, ws, st, tlev);
  ++*nl;
  TcParams prm;
  if (!common_params<F, NPASS>(P, ws, &prm)) return cudaErrorInvalidValue;
  prm.accumulate = 1;  // P2L over X adds into the same expansions
  if (prm.ncls != 1) {  // gathered rows belong to one class: no stacked classes
    using C = Cfg<NPASS>;
    prm.ncls = 1;
    prm.stage_bytes = C::stage_bytes(prm.nc);
    prm.nstages = std::min(kMaxStages, (kSmemCap - 1024 - 256 - kBM * (int)sizeof(int)) / prm.stage_bytes);
  }
  const int ngrp = 8;
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
    const unsigned nbl = (unsigned)(t.loff[l + 1] - t.loff[l]);
    // a window less than half full is contracted over its target cells alone
    // (the source rows gathered); a fuller one in tiles of the window.  On the
    // 2M-point Plummer tree, gathering levels 7 and 8 (43% and 39% full) saved
    // 1.5 ms; level 6 (64% full, a 201 MB window beyond L2) ran 3x slower
    // per CTA gathered than in tiles.
    const bool gather = 2.0 * (double)nbl < (double)cells;
    auto a256 = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t rows = cells + (gather ? 1 : 0);  // gathered: a zero row at the end
    const size_t need = a256(rows * cell_bytes) * (NPASS == 3 ? 2 : 1) +
                        a256(cells * sizeof(int)) +
                        (gather ? a256((size_t)nbl * sizeof(int)) + 256 : 0);
    if (need > ws.tc_arena_bytes) continue;  // a window larger than the arena: CUDA cores
    if (used + need > ws.tc_arena_bytes || prm.nlev == kTcMaxLevels) {
      // contract the levels packed so far, then pack the next ones into the
      // same arena (the stream orders the packing after that launch)
      const cudaError_t e = launch_contraction<F, NPASS>(P, prm, nb, st, false);
      ++*nl;
      if (e != cudaSuccess) return e;
      prm.nlev = 0;
      nb = 0;
      used = 0;
    }
    char* at = arena + used;
    T* bhi = reinterpret_cast<T*>(at);
    at += a256(rows * cell_bytes);
    T* blo = nullptr;
    if (NPASS == 3) {
      blo = reinterpret_cast<T*>(at);
      at += a256(rows * cell_bytes);
    }
    int* map = reinterpret_cast<int*>(at);
    at += a256(cells * sizeof(int));
    int* tlist = gather ? reinterpret_cast<int*>(at) : nullptr;
    int* toff = gather ? reinterpret_cast<int*>(at + a256((size_t)nbl * sizeof(int))) : nullptr;
    used += need;
    cudaMemsetAsync(bhi, 0, rows * cell_bytes, st);
    if (blo) cudaMemsetAsync(blo, 0, rows * cell_bytes, st);
    cudaMemsetAsync(map, 0xff, cells * sizeof(int), st);
    k_apack<F><<<std::min<unsigned>((nbl + 7) / 8, 152 * 16), 256, 0, st>>>(
        t, l, ws.mp, nj, JP, W0[0], W0[1], W0[2], H[0], H[1], H[2], bhi, blo, map);
    ++*nl;
    if (gather) {
      k_alist<<<1, 1024, 0, st>>>(t, l, W0[0], W0[1], W0[2], H[0], H[1], tlist, toff);
      ++*nl;
    }
    TcLevel& v = prm.lev[prm.nlev++];
    v.l = l;
    v.l2 = 0;
    v.Hx = H[0];
    v.Hy = H[1];
    v.Hz = H[2];
    v.gather = gather ? 1 : 0;
    v.tlist = tlist;
    v.toff = toff;
    v.zero_row = (int)cells;
    v.first_block = nb;
    if (gather) {  // 128 list entries per CTA, the classes interleaved; a class holds at
                   // most one cell per parent of the window
      v.BX = 8;
      v.BY = 4;
      v.BZ = 4;
      v.ntx = v.nty = 1;
      const size_t per_cls = std::min<size_t>(nbl, cells / 8);
      nb += 8 * (int)((per_cls + kBM - 1) / kBM);
    } else {
      tile_shape(H[0], H[1], H[2], &v);
      const int ntz = (H[2] + v.BZ - 1) / v.BZ;
      nb += v.ntx * v.nty * ntz * ngrp;
    }
    v.lc = ws.lc;
    v.map = map;
    v.scale = 1.0f;
    if (shared_t) {
      const int k = l - 2;
      v.scale = pd.kernel == FMM_KERNEL_LAPLACE ? std::ldexp(1.0f, k) : std::ldexp(1.0f, -k);
    }
    if (!offset_maps<F, NPASS>(ws, shared_t ? 0 : l - 2, prm, &v)) return cudaErrorInvalidValue;
    v.ghi = reinterpret_cast<const char*>(bhi);
    v.glo = reinterpret_cast<const char*>(NPASS == 3 ? blo : bhi);
    if (!gather) {
      if (!source_map<F, NPASS>(&v.S, bhi, JP, H[0], H[1], H[2], v.BX, v.BY, v.BZ))
        return cudaErrorInvalidValue;
      v.Slo = v.S;
      if (NPASS == 3 &&
          !source_map<F, NPASS>(&v.Slo, blo, JP, H[0], H[1], H[2], v.BX, v.BY, v.BZ))
        return cudaErrorInvalidValue;
    }
    *done |= 1u << l;
  }
  if (prm.nlev == 0) return cudaGetLastError();
  const cudaError_t r = launch_contraction<F, NPASS>(P, prm, nb, st, false);
  ++*nl;
  return r;
}

}  // namespace

cudaError_t launch_m2l_tc(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st, int* nl,
                          bool tables_ready) {
  const int L = P->desc.levels;
  if (P->pd.d != 3) {
    cudaMemsetAsync(ws.lc, 0, sizeof(double) * (size_t)ws.lev_off[L + 1] * P->pd.nj, st);
    return launch_m2l_simt_levels(P, ws, 2, L, st, nl);
  }
  const int prec = P->desc.precision;
  const cudaError_t e =
      prec == FMM_PREC_F16X3    ? run_all_levels<FmtF16, 3>(P, ws, st, tables_ready)
      : prec == FMM_PREC_BF16X3 ? run_all_levels<FmtBF16, 3>(P, ws, st, tables_ready)
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
  const int tlev = kernel_homogeneous(P->pd.kernel) ? 1 : P->desc.levels - 1;
  if (prec == FMM_PREC_F16X3) build_tables<FmtF16, 3>(P, ws, st, tlev);
  else if (prec == FMM_PREC_BF16X3) build_tables<FmtBF16, 3>(P, ws, st, tlev);
  else if (prec == FMM_PREC_TF32X3) build_tables<FmtTF32, 3>(P, ws, st, tlev);
  else build_tables<FmtTF32, 1>(P, ws, st, tlev);
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
