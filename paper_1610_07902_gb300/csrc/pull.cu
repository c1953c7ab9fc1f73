// Pull direction (matrix-driven SpMSpV, Sec. II-B): not yet available.
#include "handle.cuh"

namespace spmspv {

int run_pull_if_available(spmspv_handle*, int, const int32_t*, const uint32_t*, int,
                          const uint32_t*, int, const Sched&, int32_t*, uint32_t*, int32_t,
                          int32_t*, cudaStream_t) {
  return -1;
}

void release_extras(spmspv_handle* h) {
  cudaFree(h->xbits);
  cudaFree(h->xdense);
  cudaFree(h->pull_status);
  cudaFree(h->bfs_front);
  cudaFree(h->bfs_visited);
  cudaFree(h->bfs_count);
}

}  // namespace spmspv
