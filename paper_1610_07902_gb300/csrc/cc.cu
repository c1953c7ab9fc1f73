// Connected components by minimum-label propagation, one masked-free
// (select2nd, min) SpMSpV per round: Sec. I names connected components among
// the graph algorithms whose workhorse is SpMSpV (the paper gives no
// algorithm; this is the plain label-propagation reading).
//
//   label(v) = v; x = {(v, v) : all v}
//   round:  y = A (min.select2nd) x       y(i) = smallest label among the
//                                         neighbours of i that changed last round
//           for (i, l) in y with l < label(i):  label(i) = l, (i, l) joins x
//   until x is empty; then label(v) = the smallest vertex id of v's component.
//
// Only the vertices whose label dropped in the last round send (a frontier),
// so the work of a round is the degree sum of that frontier.  The rounds run
// as one CUDA graph: a WHILE node whose body is K1 -> K2 -> K3 on the
// frontier, the label update, and the loop condition.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "handle.cuh"
#include "spmspv_internal.cuh"

namespace spmspv {
namespace {

__global__ void k_cc_init(int32_t n, int32_t* __restrict__ labels, int32_t* __restrict__ x_idx,
                          uint32_t* __restrict__ x_val, int32_t* __restrict__ cnt, DevState* st) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    labels[v] = v;
    x_idx[v] = v;
    x_val[v] = (uint32_t)v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    cnt[0] = n;  // this round's frontier
    cnt[1] = 0;  // the next round's, appended by the update
    st->level = 0;
    st->cc_labels = labels;
  }
}

// The round's y: lower labels win, their vertices form the next frontier.
__global__ void k_cc_update(const DevState* __restrict__ st, const int32_t* __restrict__ y_idx,
                            const uint32_t* __restrict__ y_val, int32_t* __restrict__ x_idx,
                            uint32_t* __restrict__ x_val, int32_t* __restrict__ cnt) {
  int32_t* const labels = st->cc_labels;
  const int32_t ny = st->nnz_y;
  const int lane = threadIdx.x & 31;
  // grid-stride in whole warps so that every lane of a warp takes part in the ballot
  for (int32_t k0 = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; k0 < ny;
       k0 += gridDim.x * blockDim.x) {
    const int32_t k = k0 + lane;
    int32_t i = 0;
    uint32_t l = 0u;
    bool lower = false;
    if (k < ny) {
      i = y_idx[k];
      l = y_val[k];
      lower = (int32_t)l < labels[i];
    }
    const unsigned b = __ballot_sync(0xffffffffu, lower);
    int32_t base = 0;
    if (lane == 0 && b) base = atomicAdd(&cnt[1], __popc(b));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (lower) {
      labels[i] = (int32_t)l;  // every i appears once in y
      const int32_t pos = base + __popc(b & ((1u << lane) - 1u));
      x_idx[pos] = i;
      x_val[pos] = l;
    }
  }
}

__global__ void k_cc_continue(cudaGraphConditionalHandle cond, DevState* st, int32_t* cnt, int32_t n) {
  if (threadIdx.x == 0) {
    cnt[0] = cnt[1];
    cnt[1] = 0;
    st->level += 1;
    cudaGraphSetConditional(cond, (cnt[0] > 0 && st->level <= n) ? 1u : 0u);
  }
}

}  // namespace

static int cc_round_launches(spmspv_handle* h, const Sched& sc, cudaGraphConditionalHandle cond,
                             cudaStream_t s) {
  int rc = graph_spmspv(h, kMinSelect2nd, sc, h->cc_x_idx, h->cc_x_val, h->cc_cnt, nullptr, h->cc_y_idx,
                        h->cc_y_val, s);
  if (rc != SPMSPV_OK) return rc;
  k_cc_update<<<h->sm_count * 4, 256, 0, s>>>(h->ws.st, h->cc_y_idx, h->cc_y_val, h->cc_x_idx,
                                               h->cc_x_val, h->cc_cnt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "cc update");
  k_cc_continue<<<1, 32, 0, s>>>(cond, h->ws.st, h->cc_cnt, h->A.n);
  return (e = cudaGetLastError()) == cudaSuccess ? SPMSPV_OK : cuda_fail(e, "cc condition");
}

void release_cc(spmspv_handle* h) {
  for (int i = 0; i < SPMSPV_NUM_SCHEDULES / 2; ++i) {
    if (h->cc_graph[i]) cudaGraphExecDestroy((cudaGraphExec_t)h->cc_graph[i]);
    h->cc_graph[i] = nullptr;
  }
  cudaFree(h->cc_x_idx);
  cudaFree(h->cc_x_val);
  cudaFree(h->cc_y_idx);
  cudaFree(h->cc_y_val);
  cudaFree(h->cc_cnt);
  h->cc_x_idx = nullptr;
  h->cc_x_val = nullptr;
  h->cc_y_idx = nullptr;
  h->cc_y_val = nullptr;
  h->cc_cnt = nullptr;
}

}  // namespace spmspv

using namespace spmspv;

extern "C" int spmspv_cc(spmspv_handle* h, int32_t* labels, int32_t* d_nrounds, uint32_t opts,
                         spmspv_stream_t stream) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (h->A.m != h->A.n) return fail(SPMSPV_ERR_ARG, "connected components need a square matrix");
  if (!(h->flags & SPMSPV_CSC_PATTERN_SYMMETRIC))
    return fail(SPMSPV_ERR_ARG, "connected components need a pattern-symmetric (undirected) matrix");
  if (!labels) return fail(SPMSPV_ERR_ARG, "labels is NULL");
  if (opts & SPMSPV_SCHED_AUTO) return fail(SPMSPV_ERR_UNSUPPORTED, "connected components run a fixed push schedule");
  int sched = h->default_sched;
  if (opts & SPMSPV_SCHED_FORCE) sched = (int)SPMSPV_SCHED_ID(opts);
  if (sched < 0 || sched >= SPMSPV_NUM_SCHEDULES / 2)
    return fail(SPMSPV_ERR_ARG, "connected components take a push schedule (0..5)");
  const size_t n = (size_t)h->A.n;
  if (!h->cc_x_idx) {
    cudaError_t e = cudaMalloc(&h->cc_x_idx, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&h->cc_x_val, sizeof(uint32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&h->cc_y_idx, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&h->cc_y_val, sizeof(uint32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&h->cc_cnt, sizeof(int32_t) * 4);
    if (e != cudaSuccess) {
      release_cc(h);
      cudaGetLastError();
      return fail(SPMSPV_ERR_OOM, "connected-component buffers: %s", cudaGetErrorString(e));
    }
  }
  if (!h->cc_graph[sched]) {
    cudaGraphExec_t exec = nullptr;
    const Sched sc = decode_schedule(h, sched);
    rc = build_while_graph(h, [&](cudaGraphConditionalHandle c, cudaStream_t cs) {
      return cc_round_launches(h, sc, c, cs);
    }, &exec);
    if (rc != SPMSPV_OK) return rc;
    h->cc_graph[sched] = exec;
  }
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  h->last_empty = 0;
  const int grid = std::max(1, std::min(h->sm_count * 8, (h->A.n + 255) / 256));
  k_cc_init<<<grid, 256, 0, s>>>(h->A.n, labels, h->cc_x_idx, h->cc_x_val, h->cc_cnt, h->ws.st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "cc init");
  if ((e = cudaGraphLaunch((cudaGraphExec_t)h->cc_graph[sched], s)) != cudaSuccess)
    return cuda_fail(e, "cc graph launch");
  if (d_nrounds) {
    e = cudaMemcpyAsync(d_nrounds, &h->ws.st->level, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "cc round count");
  }
  return SPMSPV_OK;
}
