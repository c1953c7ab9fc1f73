// Learned schedule selector (placeholder until the network is added).
#include <cuda_runtime.h>

#include "handle.cuh"

namespace spmspv {
cudaError_t launch_selector(spmspv_handle* h, int allow_pull, cudaStream_t s) {
  (void)h;
  (void)allow_pull;
  (void)s;
  return cudaErrorNotSupported;
}
}  // namespace spmspv
