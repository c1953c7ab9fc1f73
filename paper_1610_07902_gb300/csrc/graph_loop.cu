// Device-side loops of the graph algorithms built on SpMSpV (connected
// components, independent sets, matching): one CUDA graph whose WHILE node
// repeats a captured body until a kernel of the body clears the condition,
// and the push SpMSpV (K1 -> K2 -> K3) such a body runs on a device-sized x.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "handle.cuh"
#include "spmspv_internal.cuh"

namespace spmspv {

int graph_spmspv(spmspv_handle* h, int sem, const Sched& sc, const int32_t* x_idx,
                 const uint32_t* x_val, const int32_t* f_dev, const uint32_t* skip_rows,
                 int32_t* y_idx, uint32_t* y_val, cudaStream_t s) {
  cudaError_t e = launch_k1(sem, h->A, h->ws, h->nb_fine, x_idx, x_val, 0, f_dev, h->k1_grid_dev, &sc, s);
  if (e != cudaSuccess) return cuda_fail(e, "work scan");
  if ((e = launch_k2(sem, h->A, h->ws, h->lwb_lo, h->nb_fine, skip_rows, 1, h->k2_grid, h->k2_smem, s,
                     0, sc.q)) != cudaSuccess)
    return cuda_fail(e, "expand/scatter");
  const int nb = (int)(((int64_t)h->A.m + (1 << sc.lwb) - 1) >> sc.lwb);
  const int k3_grid = std::max(1, std::min(nb, h->sm_count * h->k3_bps[sc.lwb - h->lwb_lo]));
  if ((e = launch_k3(sem, false, h->A, h->ws, h->lwb_lo, h->nb_fine, y_idx, y_val, h->A.m, nullptr,
                     nullptr, k3_grid, k3_smem_bytes(sc.lwb), s)) != cudaSuccess)
    return cuda_fail(e, "merge");
  return SPMSPV_OK;
}


int build_while_graph(spmspv_handle* h,
                      const std::function<int(cudaGraphConditionalHandle, cudaStream_t)>& body,
                      cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
  int rc = SPMSPV_OK;
  do {
    cudaGraphConditionalHandle cond;
    if ((e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess) {
      rc = cuda_fail(e, "loop condition handle");
      break;
    }
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np)) != cudaSuccess) {
      rc = cuda_fail(e, "loop while node");
      break;
    }
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) {
      rc = cuda_fail(e, "capture stream");
      break;
    }
    if ((e = cudaStreamBeginCaptureToGraph(cs, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
      rc = cuda_fail(e, "begin capture");
      break;
    }
    void* saved_prof = h->prof;
    h->prof = nullptr;
    rc = body(cond, cs);
    h->prof = saved_prof;
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(cs, &captured);
    if (rc != SPMSPV_OK) break;
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "end capture");
      break;
    }
    if ((e = cudaGraphInstantiate(&exec, g, 0)) != cudaSuccess) rc = cuda_fail(e, "instantiate loop graph");
  } while (0);
  if (cs) cudaStreamDestroy(cs);
  cudaGraphDestroy(g);
  if (rc != SPMSPV_OK) {
    if (exec) cudaGraphExecDestroy(exec);
    cudaGetLastError();
    return rc;
  }
  *out = exec;
  return SPMSPV_OK;
}

}  // namespace spmspv
