// fmm_eval_noalloc: the FMM evaluation with its workspace taken from a fixed
// array that the library reserves statically on every device it is loaded
// on, so the call itself allocates nothing.
//
// Who needs this: callers that are not allowed to allocate device memory at
// the point where they evaluate -- for example code that runs while a CUDA
// stream is being captured into a graph (allocation is not a capturable
// operation), real-time loops that forbid allocation after start-up, or
// plug-ins living inside a host framework that owns the whole memory pool.
// They pay with a fixed size limit and with a shared buffer (see ctfmm.h).
#include <mutex>

#include "fmm_internal.cuh"

// 32 MiB, aligned for the workspace layout (256 B).  Held by every device that
// loads the library until the process exits.
#define FMM_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[FMM_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};

// Device address of the scratch array for the current device, looked up once
// per device with that device current.  In host code the array's name is
// only a host-side stand-in, never a device address.
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FMM_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return FMM_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return FMM_ERR_CUDA;
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return FMM_OK;
}

}  // namespace

extern "C" int fmm_eval_noalloc(fmm_plan_t plan, int64_t n_src, const double* src_dev,
                                const double* w_dev, int64_t n_tgt, const double* tgt_dev,
                                double* phi_dev, double* grad_dev, void* stream) {
  if (!plan) return FMM_ERR_ARG;
  size_t need = 0;
  const int rc = fmm_workspace_size(plan, n_src, n_tgt, &need);
  if (rc != FMM_OK) return rc;
  if (need > FMM_NOALLOC_SCRATCH_BYTES) return FMM_ERR_WORKSPACE;
  if (n_tgt > 0 && !phi_dev) return FMM_ERR_ARG;  // the same check as fmm_eval
  void* scratch = nullptr;
  const int rs = scratch_address(&scratch);
  if (rs != FMM_OK) return rs;
  return fmm_eval(plan, n_src, src_dev, w_dev, n_tgt, tgt_dev, phi_dev, grad_dev, scratch,
                  FMM_NOALLOC_SCRATCH_BYTES, stream);
}
