// Internal declarations shared by the CUDA translation units of libctfmm.
//
// Coefficient layouts (all multi-index tables are built by plan.cu):
//  * "Full" layout of M(P): slabs by the slow (last) exponent m_s = 0..P;
//    inside a slab (d=3) rows by m_1, each row m_0 = 0..P-m_s-m_1.  The
//    position of (m_0, m_1, m_s) is row_base[m_s][m_1] + m_0.
//  * The stored set j = {m : m_s < c} (Lemma 5 with the last axis slowest) is
//    therefore the PREFIX of the full layout: its first nj entries.
//  * "Hankel" layout: the same slab layout for order 2p, slabs 0..2c-2 only:
//    exactly the derivatives d^{i+q} G with i, q in j that M2L reads
//    (eq. (m2l_toeplitz)).
// Expansions are stored box-scaled: at level l with box side s_l,
//   multipole  bt_q = beta_q / s^{|q|},    local  Lt_i = s^{|i|} L_i,
// so that derivatives are taken in units of the box side (this only scales
// the coefficients; eqs. of Secs. 3-4 are unchanged).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ctfmm.h"

#define FMM_MAXP 20

// Kernel ids inside the device code.  A Helmholtz plan (G = e^{i kappa r}/r)
// is evaluated as two real FMMs that share the tree, P2M and M2M -- the
// multipoles are real for real weights and the PDE Laplacian + kappa^2 has
// real coefficients -- one with the real part cos(kappa r)/r (kernel id
// FMM_KERNEL_HELMHOLTZ) and one with the imaginary part sin(kappa r)/r
// (kHelmIm); their potentials are the real and imaginary parts of phi.
constexpr int kHelmIm = 16;
// kernels whose derivatives come from the coupled (g, b) recurrence:
// r^2 d_a g = -x_a g + alpha x_a b, d_a b = beta x_a g
__host__ __device__ inline bool kernel_screened(int k) {
  return k == FMM_KERNEL_YUKAWA || k == FMM_KERNEL_HELMHOLTZ || k == kHelmIm;
}
// the precisions whose dense M2L runs on the tensor cores (3D)
__host__ __device__ inline bool prec_tensor(int prec) {
  return prec == FMM_PREC_TF32 || prec == FMM_PREC_TF32X3 || prec == FMM_PREC_BF16X3 ||
         prec == FMM_PREC_F16X3;
}
// G(s h) = s^deg G(h): one set of M2L tables serves every level
__host__ __device__ inline bool kernel_homogeneous(int k) {
  return k == FMM_KERNEL_LAPLACE || k == FMM_KERNEL_BIHARMONIC;
}
#define FMM_MAX_TERMS 12
#define FMM_MAX_LEVELS 8

// Geometry of the root box, resident in device memory (written per call).
struct Geom {
  double lo[3];
  double size;
  double s_leaf;      // size / 2^L
  double inv_s_leaf;  // 1 / s_leaf
  int flag;  // device-side status bits (1: domain, 2: timeout, 4: traversal stack full)
  int pad;
  unsigned long long m2l_count;  // adaptive trees: M2L translations performed
  unsigned long long p2p_pairs;  // uniform trees, when timing: near-field pairs
};

// Read-only plan data passed by value to kernels.
struct PlanDev {
  int d, p, c;
  int nfull;  // N(p)
  int nj;     // |j|
  int nh;     // entries of the Hankel layout (order 2p, slabs 0..2c-2)
  int kernel;
  double lam;
  int nterms;                      // decompression recurrence terms
  int tsh[FMM_MAX_TERMS][3];       // shift xi - c e_s  (d=2 uses [0],[1])
  double tcoef[FMM_MAX_TERMS];     // -a_xi / a_{c e_s}
  float tcoef_f[FMM_MAX_TERMS];    // the same rounded to float (float kernels, tpow = 0)
  int tpow[FMM_MAX_TERMS];         // c - |xi|: power of s_l in the scaled coefficient
  // device tables
  const char4* mi;         // nfull: (m0, m1, m2, |m|); d=2 uses (m0, m_s, 0, |m|)
  const double* inv_fact;  // nfull: 1/m!
  const float* inv_fact_f; // nfull: 1/m! rounded to float (float kernels: no FP64 work)
  const float* fact_f;     // nfull: m! (sqrt 2)^|m| rounded to float (m! = m_0! m_1! m_2!),
                           // the F16X3 operand scale (its offset matrices divide by it)
  const int16_t* rec_src;  // nfull x nterms: decompression sources (rows with m_s >= c)
  const int16_t* cmp_src;  // nfull x nterms: compression gather sources (-1 = none)
  const int* frow;         // full layout row bases:   [m_s*(p+1) + m_1]   (d=2: [m_s])
  const int* hrow;         // Hankel layout row bases: [m_s*(2p+1) + m_1]  (d=2: [m_s])
  // P2M monomial segments (d = 3): runs of up to 4 consecutive m_0 of one row
  // of the full layout, packed m_0 | m_1 << 5 | m_s << 10 | len << 15 | pos << 18
  const int* p2m_seg;
  int p2m_nseg;
};

// Transform sizes and tables of the FFT form of M2L (eq. (convolution_m2l)).
// Axis a of the coefficient grid (a = 0: m_0, 1: m_1 (d = 3), 2: m_s) has
// length n_a = 2 M_a + 1 with M = (p, p, c - 1) (d = 2: (p, 1, c - 1)); the
// spectra keep the Hermitian half k_0 = 0..p of the m_0 axis.
struct FftDev {
  int n1, n2, n3;      // transform lengths along m_0, m_1 (1 when d = 2), m_s
  int k1;              // p + 1 stored frequencies along m_0
  int kf;              // k1 * n2 * n3 complex values per spectrum
  int kfp;             // kf rounded up to a multiple of 32 (row stride)
  const double* tw1;   // n1 x (cos, sin)(2 pi n / n1); also serves axis 1 (n2 = n1 or 1)
  const double* tw3;   // n3 x (cos, sin)(2 pi n / n3)
  const double* gpow;  // g^n and g^-n, n = 0..2p (2 x (2p + 1))
};

struct fmm_plan_s {
  fmm_plan_desc desc;
  PlanDev pd;
  FftDev fft;
  void* dev_tables;
  int timing;
  cudaEvent_t ev[FMM_NUM_PHASES + 1];
  cudaEvent_t evk[2];  // around the M2L contraction launch(es)
  bool events_made;
  // FP32 3D uniform path: the pipeline on a high-priority stream, the M2L
  // tables and the near field on a low-priority one; events order them after
  // the caller's stream (in), the tables and near field after the sort (fork),
  // the M2L after the tables (tab), the far field after the near field (join)
  // and the caller's stream after the pipeline (out)
  cudaStream_t hi, aux;
  cudaEvent_t ev_in, ev_fork, ev_join, ev_out;
  cudaEvent_t ev_tab;  // derivative and offset tables built (on aux)
  cudaStream_t last_stream;
  Geom* last_geom;  // device geometry of the last evaluation (in its workspace)
  int launches;
  int deriv_levels;  // adaptive plans: M2L table levels of the current tree
  int last_boxes;    // adaptive plans: boxes and depth of the last tree
  int last_depth;
  // adaptive plans: per level l, the smallest (6l + k) and largest (6l + 3 + k)
  // coordinate k of the last tree's boxes, read with its level offsets
  int abnd[6 * (16 + 2)];
  long long tc_wait_cycles;  // tensor-core M2L pipeline waits (0: the default ~1 s)
};

inline void set_deriv_levels(const fmm_plan_s* P, int maxlev) {
  const_cast<fmm_plan_s*>(P)->deriv_levels = maxlev;
}

// record the start (i = 0) or end (i = 1) of the M2L contraction when timing
inline void mark_contraction(const fmm_plan_s* P, int i, cudaStream_t st) {
  if (P->timing) cudaEventRecord(P->evk[i], st);
}

// ---------------------------------------------------------------------------
// Workspace layout of one evaluation.
// ---------------------------------------------------------------------------
struct Workspace {
  Geom* geom;
  // points, sorted by leaf box (SoA)
  double* sx[3];
  double* sw;
  int* sperm;       // sorted position -> original source index
  double* tx[3];
  int* tperm;       // sorted position -> original target index
  int* sstart;      // nleaf + 1
  int* tstart;      // nleaf + 1
  // radix sort scratch
  uint32_t* keys_a;
  uint32_t* keys_b;
  int* vals_a;
  int* vals_b;
  int* hist;        // 256 x nblocks
  int* hist_sums;   // chunk sums
  int* counts;      // nleaf
  // expansions (levels 2..L), box-scaled, float64
  double* mp;       // sum_l nbox(l) * nj
  double* lc;
  int64_t lev_off[FMM_MAX_LEVELS + 1];  // offset (in boxes) of level l inside mp/lc
  // M2L derivative tables: (L-1) levels x 7^d offsets x nh
  double* htab;
  // bounding-box reduction scratch
  double* bbox;     // 2*d*nblocks
  int nbbox_blocks;
  // tensor-core M2L operands (tf32 hi / lo): parity-split multipoles of the
  // finest level and the dense offset matrices of one level
  int tc_jp;        // |j| padded to one K chunk of the operand format (row length)
  int tc_mp;        // rows of one offset matrix: |j| padded to the column blocks (tc_shape)
  void* tc_bpar[2];
  void* tc_tmat[2];
  float* tc_bscale;  // F16X3: the power of two each box's packed multipole was divided by
  // adaptive trees: arena for the per-level windows (parity-split operands
  // and cell -> box maps) and the per-level coordinate bounds
  void* tc_arena;
  size_t tc_arena_bytes;
  // FFT form of M2L: spectra of the multipoles and of the local sums of every
  // box of levels 2..L (kfp complex each) and of the offset tables
  void* fft_b;
  void* fft_g;
  void* fft_h;
  // FP32 leaf path: box-relative coordinates (x - c_own)/s and weight, and the
  // decompressed far-field coefficients M Lt / m! of every leaf
  float4* sxr;
  float4* txr;
  // adaptive tree (plans with levels < 0): box arrays of capacity anb_cap and
  // the points' Morton codes in sorted order
  int64_t anb_cap;
  uint32_t* akey;
  int* alev;
  int* apar;
  int* achild;
  int* as0;
  int* as1;
  int* at0;
  int* at1;
  int* aleaf;
  unsigned char* am2p;  // per box: a leaf with W boxes of more than |j| sources (float pass)
  // float leaf pass: the sorted sources as two floats per coordinate, hi = fl(x)
  // (and the weight) and lo = fl(x - hi), so that box-relative coordinates
  // need no FP64 arithmetic (null in the FP64 mode)
  float4* asxh;
  float4* asxl;
  int* aloff;           // tree build: level offsets on the device, the overflow flag, the
                        // per-level coordinate bounds
  int* anch;
  int* ascan;
  uint32_t* skey;
  uint32_t* tkey;
  int* agrid;       // dense box index of the coarse levels (adaptive.cuh)
  // Helmholtz plans: potentials (2 x n_tgt) and gradients (2 x d x n_tgt) of
  // the real and the imaginary part
  double* hphi;
  double* hgrad;
  size_t bytes;
};

// helpers
__host__ __device__ inline int64_t nbox_at(int d, int l) { return (int64_t)1 << (d * l); }

// Blocking of the tensor-core M2L contraction (m2l_tc.cu).  The MMA's M
// dimension holds 128 target boxes, N the local coefficients i of j and K the
// multipole coefficients q.  |j| is padded to a multiple of 16 (the MMA's N
// granularity) and split into nchunk column blocks of nc <= 256 columns; when
// one block of nc columns leaves room, ncls child classes of the target boxes
// share one CTA (their offset matrices stacked along N, up to 256 columns).
// Rows of the operands are jp = |j| padded to a whole K chunk of row_bytes
// (128 bytes).
struct TcShape {
  int row_bytes, esz, jp;
  int nc, nchunk, npt, ncls;
};
inline TcShape tc_shape(int nj, int precision) {
  TcShape s;
  s.row_bytes = 128;
  s.esz = (precision == FMM_PREC_BF16X3 || precision == FMM_PREC_F16X3) ? 2 : 4;
  const int row = s.row_bytes / s.esz;
  s.jp = (nj + row - 1) / row * row;
  const int nj16 = (nj + 15) / 16 * 16;
  s.nchunk = (nj16 + 255) / 256;
  s.nc = ((nj16 + s.nchunk - 1) / s.nchunk + 15) / 16 * 16;
  s.npt = s.nchunk * s.nc;
  s.ncls = 1;
  if (s.nchunk == 1)
    while (s.ncls < 8 && 2 * s.ncls * s.nc <= 256) s.ncls *= 2;
  return s;
}

int fmm_workspace_layout(const fmm_plan_s* P, int64_t n_src, int64_t n_tgt, void* base,
                         Workspace* ws);

// launchers (defined in the .cu files); each returns cudaGetLastError()
cudaError_t launch_set_geom(const fmm_plan_s* P, const Workspace& ws, int64_t n_src,
                            const double* src, int64_t n_tgt, const double* tgt,
                            cudaStream_t st, int* nlaunch);
cudaError_t launch_build_tree(const fmm_plan_s* P, const Workspace& ws, int64_t n_src,
                              const double* src, const double* w, int64_t n_tgt,
                              const double* tgt, cudaStream_t st, int* nlaunch);
cudaError_t launch_deriv_tables(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st,
                                int* nlaunch);
cudaError_t launch_p2m(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st, int* nlaunch);
cudaError_t launch_m2m(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st, int* nlaunch);
// tables_ready: launch_m2l_tables has already been ordered before this call
cudaError_t launch_m2l(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st, int* nlaunch,
                       bool tables_ready = false);
cudaError_t launch_m2l_tables(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st,
                              int* nlaunch);
cudaError_t launch_m2l_fft(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st,
                           int* nlaunch);
// offset tables of the M2L derivative tables: one level suffices when the
// kernel is homogeneous (3D Laplace, biharmonic) and the M2L path rescales
bool m2l_shared_tables(const fmm_plan_s* P);
cudaError_t launch_l2l(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st, int* nlaunch);
cudaError_t launch_leaf_eval(const fmm_plan_s* P, const Workspace& ws, double* phi,
                             double* grad, cudaStream_t st, int* nlaunch);
bool leaf_split_supported(const fmm_plan_s* P);
cudaError_t launch_near_field(const fmm_plan_s* P, const Workspace& ws, double* phi,
                              double* grad, cudaStream_t st, int* nlaunch);
cudaError_t launch_far_field(const fmm_plan_s* P, const Workspace& ws, double* phi,
                             double* grad, cudaStream_t st, int* nlaunch);

// adaptive tree (adaptive.cuh): the build synchronises the stream once per
// level to size the next level; *tree receives the level offsets
struct ATree;
cudaError_t launch_build_adaptive(const fmm_plan_s* P, const Workspace& ws, int64_t n_src,
                                  const double* src, const double* w, int64_t n_tgt,
                                  const double* tgt, cudaStream_t st, int* nlaunch,
                                  ATree* tree, int* overflow);
cudaError_t launch_adaptive_upward(const fmm_plan_s* P, const Workspace& ws, const ATree& t,
                                   cudaStream_t st, int* nlaunch);
cudaError_t launch_adaptive_m2l(const fmm_plan_s* P, const Workspace& ws, const ATree& t,
                                cudaStream_t st, int* nlaunch);
// tensor-core M2L of an adaptive tree (levels packed into dense windows);
// levels whose window does not fit the arena are left to the caller
// (*done_mask bit l set for every level handled)
cudaError_t launch_adaptive_m2l_tc(const fmm_plan_s* P, const Workspace& ws, const ATree& t,
                                   cudaStream_t st, int* nlaunch, unsigned* done_mask);
cudaError_t launch_adaptive_p2l_l2l(const fmm_plan_s* P, const Workspace& ws, const ATree& t,
                                    cudaStream_t st, int* nlaunch);
cudaError_t launch_adaptive_leaf_warp(const fmm_plan_s* P, const Workspace& ws, const ATree& t,
                                      double* phi, cudaStream_t st, int* nlaunch);
cudaError_t launch_adaptive_leaf(const fmm_plan_s* P, const Workspace& ws, const ATree& t,
                                 double* phi, cudaStream_t st, int* nlaunch);
