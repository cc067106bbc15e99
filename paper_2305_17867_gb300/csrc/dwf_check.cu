// fmm_selftest_dw: the double-word float operations of dwf.cuh applied to
// host arrays, so that tests can hold them to their error bounds.
#include <vector>

#include "../../include/ctfmm.h"
#include "dwf.cuh"

namespace {

__global__ void k_dw_ops(int op, int64_t n, const double* __restrict__ x,
                         const double* __restrict__ y, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const dwf a(x[i]), b(y[i]);
  const dwf r = op == 0 ? a + b : op == 1 ? a * b : fma(a, b, a);
  out[i] = (double)r;
}

}  // namespace

extern "C" int fmm_selftest_dw(int op, int64_t n, const double* x, const double* y, double* out) {
  if (op < 0 || op > 2 || n < 0 || (n > 0 && (!x || !y || !out))) return FMM_ERR_ARG;
  if (n == 0) return FMM_OK;
  double* d = nullptr;
  const size_t bytes = sizeof(double) * (size_t)n;
  if (cudaMalloc(&d, 3 * bytes) != cudaSuccess) return FMM_ERR_CUDA;
  bool ok = cudaMemcpy(d, x, bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(d + n, y, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
  if (ok) {
    k_dw_ops<<<(unsigned)((n + 255) / 256), 256>>>(op, n, d, d + n, d + 2 * n);
    ok = cudaGetLastError() == cudaSuccess &&
         cudaMemcpy(out, d + 2 * n, bytes, cudaMemcpyDeviceToHost) == cudaSuccess;
  }
  cudaFree(d);
  return ok ? FMM_OK : FMM_ERR_CUDA;
}
