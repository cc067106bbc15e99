/*
 * ctfmm.h -- C ABI of the GB300 compressed-Taylor FMM.
 *
 * Method: Fernando & Kloeckner, "Automatic Synthesis of Low-Complexity
 * Translation Operators for the Fast Multipole Method" (arXiv 2305.17867).
 * The library evaluates the many-body potential of eq. (1),
 *     phi(x) = sum_{y in S, y != x} G(x - y) w(y),   x in T,
 * with a Taylor FMM on a uniform or an adaptive tree whose expansions are
 * stored compressed by the PDE that G satisfies (Sec. 3): only the
 * multi-indices j = {m in M(p):
 * m_d < c} are kept (Lemma 5, last axis slowest), derivatives of G come from
 * r^2-led recurrences (Sec. 4.4), and every stage -- tree build, P2M, M2M,
 * M2L, L2L, L2P, P2P -- runs as CUDA kernels on the caller's stream.
 *
 * Conventions for every entry point:
 *  - Pointers named *_dev are DEVICE pointers (cudaMalloc'd or torch tensors
 *    on the current device).  Points are row-major n x d float64 arrays.
 *  - All device work is enqueued on the `stream` argument (a cudaStream_t,
 *    NULL = legacy default stream).  Calls return as soon as the work is
 *    enqueued; nothing is synchronised except where stated.  Uniform 3D
 *    plans of the float precisions run the pipeline on two streams the plan
 *    owns (the M2L tables and the near field on a low-priority one,
 *    concurrently with the rest on a high-priority one), joined to `stream`
 *    by events on both sides: to the caller the work is still ordered on
 *    `stream`, and a call made while `stream` is being captured into a CUDA
 *    graph captures both branches.
 *  - The caller owns every input, output and workspace buffer.  The library
 *    owns the plan and the small read-only tables the plan uploads at
 *    creation (cudaMalloc'd once, freed by fmm_plan_destroy).
 *  - Return values are fmm_status codes (0 = success, negative = error).
 *    Nothing is printed and no exception crosses the ABI.
 *  - A plan is not thread-safe: calls that use the same plan must not run
 *    concurrently, and evaluations sharing one workspace must be ordered on
 *    the GPU (one stream, or events).
 */
#ifndef CTFMM_H
#define CTFMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmm_plan_s* fmm_plan_t;

typedef enum {
  FMM_OK = 0,
  FMM_ERR_ARG = -1,          /* invalid argument (null pointer, bad size or enum) */
  FMM_ERR_UNSUPPORTED = -2,  /* kernel/dimension/PDE combination not provided */
  FMM_ERR_CUDA = -3,         /* a CUDA runtime call failed */
  FMM_ERR_NOMEM = -4,        /* plan tables could not be allocated */
  FMM_ERR_TIMEOUT = -5,      /* a bounded device wait gave up */
  FMM_ERR_DOMAIN = -6,       /* a point lay outside the root box (it was clamped) */
  FMM_ERR_WORKSPACE = -7,    /* workspace too small */
  FMM_ERR_INCOMPLETE = -8    /* a fixed-size device structure overflowed: the result
                                is incomplete (reported by fmm_last_status) */
} fmm_status;

/* Kernels G (reading of the paper's normalisations):
 *  LAPLACE     d=2: log|x|            d=3: 1/(4 pi |x|)     PDE: Laplacian
 *  YUKAWA      d=3: exp(-lambda |x|)/|x|                    PDE: Laplacian - lambda^2
 *  BIHARMONIC  d=2: |x|^2 log|x|     d=3: |x|              PDE: Laplacian^2
 *  HELMHOLTZ   d=3: exp(i kappa |x|)/|x|, kappa = the `lambda` field
 *                                                           PDE: Laplacian + kappa^2
 * A Helmholtz potential is complex: phi_dev (and grad_dev) then hold complex
 * values, real and imaginary parts interleaved (2 doubles per value). */
enum {
  FMM_KERNEL_LAPLACE = 0,
  FMM_KERNEL_YUKAWA = 1,
  FMM_KERNEL_BIHARMONIC = 2,
  FMM_KERNEL_HELMHOLTZ = 3
};

/* Arithmetic of the evaluation.
 *  FP64     every stage in float64 (the parity configuration).
 *  FP32     M2L as float32 SIMT products; P2M, L2P, P2P in float32; derivative
 *           tables and the upper tree's M2M and L2L in float64 (the shifts
 *           between the leaves and their parents in float32, since their input
 *           or consumer is float32).
 *  TF32     as FP32 but M2L on the tensor cores (tcgen05 kind::tf32), one pass.
 *  TF32X3   M2L with split operands a = hi + lo in tf32, three tensor passes
 *           (hi*hi + hi*lo + lo*hi), float32 accumulation.
 *  BF16X3   the same split in bf16 (kind::f16), float32 accumulation.
 *  F16X3    the same split in fp16 (kind::f16): fp16 keeps tf32's 11-bit
 *           significand, so the products are as exact as TF32X3's, at the
 *           rate of the 16-bit tensor cores.  Its 5-bit exponent is made to
 *           suffice by scalings: with S_m = m! (sqrt 2)^|m|, each box's
 *           multipole times S_q is scaled by a power of two into [1/2, 1), the
 *           offset matrices are taken as Ht_{i+q} / (S_i S_q) over a power of
 *           two of the level's derivative scale, and the scalings are undone
 *           in float as each offset's product leaves the accumulator.  3D
 *           uniform trees only (an adaptive plan returns
 *           FMM_ERR_UNSUPPORTED).                                          */
enum {
  FMM_PREC_FP64 = 0,
  FMM_PREC_FP32 = 1,
  FMM_PREC_TF32 = 2,
  FMM_PREC_TF32X3 = 3,
  FMM_PREC_BF16X3 = 4,
  FMM_PREC_F16X3 = 5
};

/* How M2L applies the translation of eq. (m2l_toeplitz).
 *  DENSE  as a dense |j| x |j| product per (target, source) pair: the CUDA
 *         cores for FP64/FP32, the tensor cores for TF32/TF32X3/BF16X3/F16X3.
 *  FFT    in its convolution form (eq. (convolution_m2l)): every box's
 *         multipole is transformed once to a (2p+1)^{d-1} (2c-1) spectrum,
 *         each target accumulates sum_h Hhat_h * Bhat_{t-h} over its
 *         interaction list frequency by frequency, and one inverse transform
 *         per target yields its local coefficients.  Coefficients are scaled
 *         by g^{|q|} before the transform (g = 3p/8 in units of the box side;
 *         Sec. 4.1.1).  FP64 (complex double) and FP32 (complex float) only. */
enum { FMM_M2L_DENSE = 0, FMM_M2L_FFT = 1, FMM_M2L_AUTO = 2 };
/* AUTO picks by arithmetic, following measurements on GB300 (3D biharmonic,
 * L = 6, p = 4..16): FFT for FP64 (its stencil runs at ~95% of the FP64 FMA
 * rate, 5-6x fewer operations than dense) and for FP32 (CUDA-core dense
 * products are slower still); DENSE on the tensor cores for TF32, TF32X3,
 * BF16X3 and F16X3.  Adaptive plans use DENSE. */

/* A constant-coefficient PDE L = sum_t coeff[t] d^{multi_idx[t]}  (eq.
 * (define_pde_op)).  multi_idx is n_terms x d exponents.  The PDE must have
 * a nonzero coefficient on c*e_d, c its order (Property 1 on the last axis). */
typedef struct {
  int n_terms;
  const int* multi_idx;
  const double* coeff;
} fmm_pde;

typedef struct {
  int kernel;          /* FMM_KERNEL_* */
  double lambda;       /* Yukawa screening lambda, or Helmholtz wavenumber kappa
                          (> 0); ignored otherwise */
  int d;               /* 2 or 3 */
  int p;               /* expansion order, 1..24 */
  int levels;          /* > 0: leaf depth L of the uniform tree (root = 0), 2..7
                          in 3D, 2..8 in 2D;
                          < 0: adaptive tree (3D, any precision, dense M2L, not
                          Helmholtz) refined down to at most level -levels (1..10) */
  const fmm_pde* pde;  /* NULL: the kernel's own PDE */
  double root_lo[3];   /* lower corner of the root box */
  double root_size;    /* side of the root box; <= 0: bounding cube of the
                          sources and targets, found on the device per call */
  int precision;       /* FMM_PREC_* */
  int m2l;             /* FMM_M2L_*; FFT requires precision FP64 or FP32 and a
                          uniform tree; AUTO resolves to DENSE on adaptive trees */
  int max_leaf;        /* adaptive tree: a box holding more than max_leaf points
                          (sources plus targets) is split; ignored when levels > 0 */
} fmm_plan_desc;

/* Create a plan: validates the description, builds the stored set j, the
 * sparse decompression recurrence of eq. (decompression) (Thm 4), the
 * multi-index tables and uploads them (cudaMalloc + cudaMemcpy, synchronous,
 * on the current device).  *out receives the plan; on error *out = NULL. */
int fmm_plan_create(fmm_plan_t* out, const fmm_plan_desc* desc);

/* Free the plan and its device tables (synchronises the device first). */
int fmm_plan_destroy(fmm_plan_t plan);

/* Number of coefficients: nfull = N(p) = C(p+d,d), nj = |j| = N(p)-N(p-c),
 * c = PDE order.  Any pointer may be NULL. */
int fmm_plan_info(fmm_plan_t plan, int* nfull, int* nj, int* c);

/* Bytes of device workspace fmm_eval / fmm_eval_backward need for the given
 * point counts.  The workspace must be 256-byte aligned. */
int fmm_workspace_size(fmm_plan_t plan, int64_t n_src, int64_t n_tgt, size_t* bytes);

/* Evaluate phi (and, if grad_dev != NULL, grad phi) at the targets.
 * Adaptive plans (levels < 0) build the tree on the device level by level
 * and synchronise `stream` once, after the deepest level, to read the levels'
 * sizes and extents that size the later launches (so the call returns after
 * the tree is built, and it cannot be captured into a CUDA graph: made while
 * `stream` is capturing, it returns FMM_ERR_UNSUPPORTED before any work is
 * enqueued); they compute phi only (grad_dev must be
 * NULL, else FMM_ERR_UNSUPPORTED) and return FMM_ERR_WORKSPACE if the tree
 * outgrows the workspace (it cannot when the workspace has the size
 * fmm_workspace_size reports, which bounds the number of boxes).
 * Arguments:
 *   src_dev  n_src x d   source positions        (device, float64)
 *   w_dev    n_src       source weights          (device, float64)
 *   tgt_dev  n_tgt x d   target positions        (device, float64); may equal src_dev
 *   phi_dev  n_tgt       output potential        (device, float64, overwritten)
 *   grad_dev n_tgt x d   output gradient or NULL (device, float64, overwritten)
 * For FMM_KERNEL_HELMHOLTZ the outputs are complex, (re, im) interleaved:
 * phi_dev holds 2 n_tgt doubles and grad_dev n_tgt x d x 2.  The real and the
 * imaginary part of G are evaluated as two real FMMs that share the tree, P2M
 * and M2M (the multipoles are real), in one stream.
 * n_src or n_tgt may be 0.  Pairs with x == y exactly are skipped.  Points
 * outside the root box are clamped into it and flagged (FMM_ERR_DOMAIN from
 * fmm_last_status).  Asynchronous on `stream`. */
int fmm_eval(fmm_plan_t plan, int64_t n_src, const double* src_dev, const double* w_dev,
             int64_t n_tgt, const double* tgt_dev, double* phi_dev, double* grad_dev,
             void* workspace_dev, size_t workspace_bytes, void* stream);

/* fmm_eval for float32 callers: positions, weights, potentials and gradients
 * are float32 device arrays with the same shapes as in fmm_eval (complex
 * outputs of Helmholtz plans again interleaved).  The points are widened to
 * float64 on the device first -- the tree, the leaf assignment and every
 * stage then run exactly as for fmm_eval in the plan's precision -- and the
 * results are rounded to float32 at the end.  The workspace must hold
 * fmm_workspace_size_f32 bytes (the float64 copies come first). */
int fmm_workspace_size_f32(fmm_plan_t plan, int64_t n_src, int64_t n_tgt, size_t* bytes);
int fmm_eval_f32(fmm_plan_t plan, int64_t n_src, const float* src_dev, const float* w_dev,
                 int64_t n_tgt, const float* tgt_dev, float* phi_dev, float* grad_dev,
                 void* workspace_dev, size_t workspace_bytes, void* stream);

/* Reverse mode of loss = sum_i u_i phi(x_i) (no counterpart in the paper):
 *   grad_w_dev   n_src       d loss/d w_j  = sum_i u_i G(x_i - y_j)      (or NULL)
 *   grad_src_dev n_src x d   d loss/d y_j  = w_j grad psi(y_j)           (or NULL)
 *   grad_tgt_dev n_tgt x d   d loss/d x_i  = u_i grad phi(x_i)           (or NULL)
 * where psi(y) = sum_i u_i G(y - x_i) is the transposed FMM (targets as
 * sources with weights u).  grad_phi_dev (n_tgt x d, or NULL) is grad phi at
 * the targets from the forward call (fmm_eval with grad_dev): when given,
 * grad_tgt is formed from it, otherwise a second FMM evaluates grad phi.
 * Same buffer conventions as fmm_eval; the workspace must be sized with
 * fmm_workspace_size(plan, max(n_src, n_tgt), max(n_src, n_tgt)).  Uniform
 * plans of real kernels only (FMM_ERR_UNSUPPORTED for adaptive and Helmholtz
 * plans). */
int fmm_eval_backward(fmm_plan_t plan, int64_t n_src, const double* src_dev,
                      const double* w_dev, int64_t n_tgt, const double* tgt_dev,
                      const double* u_dev, const double* grad_phi_dev, double* grad_w_dev,
                      double* grad_src_dev, double* grad_tgt_dev, void* workspace_dev,
                      size_t workspace_bytes, void* stream);

/* fmm_eval without any allocation.  The paper has no counterpart; this is a
 * service for callers that may not allocate device memory when they evaluate:
 * code running while a stream is captured into a CUDA graph (allocation cannot
 * be captured), real-time loops that forbid allocation after start-up, and
 * plug-ins inside a host framework that owns the whole device memory pool.
 * Arguments and results are those of fmm_eval, minus the workspace: the
 * workspace comes from a 32 MiB array that the library reserves statically on
 * every device it is loaded on (held until the process exits).
 *  - Sizes whose fmm_workspace_size() exceeds 32 MiB are rejected with
 *    FMM_ERR_WORKSPACE before any work is enqueued (use fmm_eval for those).
 *  - Calls to cudaMalloc, cudaFree or any allocating routine: none.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current); make that first call
 *    before any stream capture begins.
 *  - Adaptive plans read level sizes back to the host while they build the
 *    tree (see fmm_eval), so they cannot run under stream capture: such a call
 *    returns FMM_ERR_UNSUPPORTED.
 *  - phi_dev must not be NULL when n_tgt > 0 (FMM_ERR_ARG, as for fmm_eval).
 *  - Every call on a device shares the one array and it keeps the previous
 *    call's contents (the evaluation clears what must start at zero itself).
 *    Calls whose GPU work overlaps -- different streams, or different plans
 *    without ordering between them -- race on the array: order them. */
int fmm_eval_noalloc(fmm_plan_t plan, int64_t n_src, const double* src_dev, const double* w_dev,
                     int64_t n_tgt, const double* tgt_dev, double* phi_dev, double* grad_dev,
                     void* stream);

/* Synchronise the stream of the last evaluation and return its device-side
 * status or a CUDA error.  Precedence: FMM_ERR_TIMEOUT (a bounded device wait
 * gave up), FMM_ERR_INCOMPLETE (an adaptive traversal stack overflowed, or any
 * status bit this version does not know), FMM_ERR_DOMAIN, FMM_OK. */
int fmm_last_status(fmm_plan_t plan);

/* Per-phase timings (milliseconds, CUDA events) of the last evaluation when
 * timing was enabled with fmm_set_timing(plan, 1); synchronises.  Phases:
 * 0 tree, 1 derivative tables, 2 P2M, 3 M2M, 4 M2L, 5 L2L, 6 L2P+P2P.
 * Where the near field runs on its own stream (see above), phase 6 is the
 * far field (leaf coefficients and L2P) plus any wait for the near field,
 * the derivative and offset tables are built on that stream too (phase 1 is
 * empty, phase 4 includes any wait for them), and the side stream's time is
 * spread over the phases it overlaps. */
#define FMM_NUM_PHASES 7
int fmm_set_timing(fmm_plan_t plan, int enable);
int fmm_phase_times(fmm_plan_t plan, float* ms_out /* FMM_NUM_PHASES */);

/* Device time (ms, CUDA events on the evaluation's stream) of the M2L
 * contraction alone -- the tensor-core launch, or the per-level SIMT launches
 * -- in the last evaluation made with timing enabled; excludes the zeroing of
 * the local expansions and the operand packing.  Synchronises. */
int fmm_m2l_kernel_time(fmm_plan_t plan, float* ms_out);

/* Tree of the last evaluation: number of boxes (all levels), deepest level
 * and number of M2L translations (interaction-list entries, List 2, summed
 * over the boxes that received them).  Uniform plans report their fixed tree;
 * for adaptive plans the count is read from the device (synchronises the
 * evaluation's stream).  Any pointer may be NULL. */
int fmm_last_tree(fmm_plan_t plan, int64_t* boxes_out, int* depth_out, int64_t* m2l_out);

/* Testing aid (no counterpart in the paper): bound the waits of the
 * tensor-core M2L's pipeline -- the TMA producer, the MMA issuer and the
 * accumulator drain -- to `cycles` SM clock cycles instead of ~1 s; 0
 * restores the default.  A wait that runs out raises the device status bit
 * that fmm_last_status reports as FMM_ERR_TIMEOUT; the kernel then waits for
 * its copies and MMAs in flight with the full limit, frees its tensor memory
 * and returns, so the context stays usable and the next evaluation (with the
 * limit restored) is unaffected. */
int fmm_set_wait_limit(fmm_plan_t plan, long long cycles);

/* Testing aid (no counterpart in the paper): the double-word float
 * arithmetic (a value held as the unevaluated sum of two floats, ~48 bits)
 * that the mixed-precision modes use for the M2M and L2L shifts above the
 * leaf level, applied elementwise on the GPU.  x, y and out are HOST arrays
 * of n doubles; each input is first rounded to a double-word float, the
 * result is converted back to double:
 *   op 0: out = x + y     op 1: out = x * y     op 2: out = x * y + x
 * Synchronous (default stream).  Returns FMM_ERR_ARG for an unknown op,
 * n < 0, or a null pointer with n > 0; FMM_ERR_CUDA on a CUDA error. */
int fmm_selftest_dw(int op, int64_t n, const double* x, const double* y, double* out);

/* Everything known about the last evaluation, in one record (synchronises
 * its stream).  Timings and the near-field pair count are filled only when
 * timing was enabled (fmm_set_timing) for that evaluation, else 0 / -1. */
typedef struct {
  float phase_ms[FMM_NUM_PHASES]; /* as fmm_phase_times */
  float m2l_kernel_ms;            /* as fmm_m2l_kernel_time */
  int64_t boxes;                  /* as fmm_last_tree */
  int depth;
  int64_t m2l_translations;
  int64_t p2p_pairs;              /* source-target pairs of the near field of a
                                     uniform tree (leaf and its 3^d - 1
                                     neighbours, coinciding points included);
                                     -1 when not counted */
  int status;                     /* as fmm_last_status */
  int launches;                   /* as fmm_last_launch_count */
} fmm_stats;
int fmm_last_stats(fmm_plan_t plan, fmm_stats* out);

/* Number of kernel launches the last fmm_eval enqueued. */
int fmm_last_launch_count(fmm_plan_t plan);

/* Human-readable text for a status code (static storage). */
const char* fmm_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* CTFMM_H */
