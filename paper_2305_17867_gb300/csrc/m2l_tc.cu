// Tensor-core M2L (tcgen05): placeholder until the kernel lands.
#include "fmm_internal.cuh"

cudaError_t launch_m2l_tc(const fmm_plan_s*, const Workspace&, cudaStream_t, int*) {
  return cudaErrorNotSupported;
}
