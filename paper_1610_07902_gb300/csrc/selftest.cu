// Failure-detection self-test: makes one bounded wait of the decoupled
// look-back run out on purpose, so that a test can see the give-up path
// report SPMSPV_DEV_TIMEOUT through the status word while the context stays
// usable (no fault, no trap, no endless loop).
#include <cuda_runtime.h>
#include <stdint.h>

#include "device_util.cuh"
#include "handle.cuh"
#include "spmspv.h"

namespace spmspv {
namespace {

// Tile 1 waits for tile 0's status word, which nothing ever publishes.
__global__ void k_wait_selftest(unsigned long long* words, DevState* st, uint32_t spins) {
  if (threadIdx.x < 32) warp_lookback(words, 1u, 1ull, st, spins);
}

}  // namespace
}  // namespace spmspv

using namespace spmspv;

extern "C" int spmspv_selftest_wait_timeout(spmspv_handle* h, uint32_t spins, spmspv_stream_t stream) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (spins < 1 || spins > SPIN_LIMIT) return fail(SPMSPV_ERR_ARG, "spins must be in [1, %u]", SPIN_LIMIT);
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* words = nullptr;
  cudaError_t e = cudaMalloc(&words, 2 * sizeof(unsigned long long));
  if (e != cudaSuccess) return fail(SPMSPV_ERR_OOM, "self-test words: %s", cudaGetErrorString(e));
  if ((e = cudaMemsetAsync(words, 0, 2 * sizeof(unsigned long long), s)) == cudaSuccess) {
    k_wait_selftest<<<1, 32, 0, s>>>(words, h->ws.st, spins);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(words);
  if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
  h->last_stream = s;
  return SPMSPV_OK;
}
