// Maximal independent set by Luby's rounds with fixed, caller-given
// priorities, two masked SpMSpVs per round.  Sec. I names maximal independent
// sets among the graph algorithms whose workhorse is SpMSpV; the paper gives
// no algorithm, so the GraphBLAS-style rounds below are this library's reading.
//
//   C = all vertices (undecided);  x = {(v, prio(v)) : v in C}
//   round:  y = A (min.select2nd) x, rows masked to C
//                      y(i) = smallest priority among the undecided neighbours of i
//           J = {v in C : v not in y, or prio(v) <= y(v)}
//                      (the local minima; equality only through a self loop)
//           in(v) = 1 for v in J;  C -= J
//           z = A (or.and) J, rows masked to C      the undecided neighbours of J
//           C -= z;  x = x restricted to C
//   until C is empty.
//
// With distinct priorities the result is the greedy set in priority order
// (the undecided vertex of smallest priority always joins, so every round
// makes progress).  The rounds run as one CUDA graph: a WHILE node whose body
// is the two SpMSpVs (K1 -> K2 -> K3 each) and the small kernels between them.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <climits>

#include "device_util.cuh"
#include "handle.cuh"
#include "spmspv_internal.cuh"

namespace spmspv {
namespace {

// cnt[0] candidates |C| (= nnz(x)), cnt[1] joiners |J|, cnt[2] survivors
__global__ void k_mis_init(int32_t n, const int32_t* __restrict__ prio, int32_t* __restrict__ in_set,
                           int32_t* __restrict__ x_idx, uint32_t* __restrict__ x_val,
                           int32_t* __restrict__ ymin, uint32_t* __restrict__ decided,
                           int32_t* __restrict__ cnt, DevState* st) {
  const int32_t nw = (n + 31) >> 5;
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    in_set[v] = 0;
    x_idx[v] = v;
    x_val[v] = (uint32_t)prio[v];
    ymin[v] = INT_MAX;
    if (v < nw) decided[v] = 0u;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    cnt[0] = n;
    cnt[1] = 0;
    cnt[2] = 0;
    st->level = 0;
    st->mis_in = in_set;
  }
}

// The first SpMSpV's y as a dense lookup (y holds undecided rows only)
__global__ void k_mis_scatter(const DevState* __restrict__ st, const int32_t* __restrict__ y_idx,
                              const uint32_t* __restrict__ y_val, int32_t* __restrict__ ymin) {
  const int32_t ny = st->nnz_y;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < ny; k += gridDim.x * blockDim.x)
    ymin[y_idx[k]] = (int32_t)y_val[k];
}

// Local minima join: membership flag, decided bit, the joiner list J.
// Every candidate's ymin entry is put back to "absent" for the next round.
__global__ void k_mis_join(const DevState* __restrict__ st, const int32_t* __restrict__ x_idx,
                           const uint32_t* __restrict__ x_val, int32_t* __restrict__ ymin,
                           uint32_t* __restrict__ decided, int32_t* __restrict__ j_idx,
                           int32_t* __restrict__ cnt) {
  int32_t* const in_set = st->mis_in;
  const int32_t nc = cnt[0];
  const int lane = threadIdx.x & 31;
  // grid-stride in whole warps so that every lane of a warp takes part in the ballot
  for (int32_t k0 = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; k0 < nc;
       k0 += gridDim.x * blockDim.x) {
    const int32_t k = k0 + lane;
    int32_t v = 0;
    bool join = false;
    if (k < nc) {
      v = x_idx[k];
      const int32_t y = ymin[v];
      ymin[v] = INT_MAX;
      join = (int32_t)x_val[k] <= y;
    }
    const int32_t pos = warp_append(join, &cnt[1]);
    if (join) {
      in_set[v] = 1;
      atomicOr(&decided[v >> 5], 1u << (v & 31));
      j_idx[pos] = v;
    }
  }
}

// The second SpMSpV's rows (undecided neighbours of J) leave C
__global__ void k_mis_remove(const DevState* __restrict__ st, const int32_t* __restrict__ z_idx,
                             uint32_t* __restrict__ decided) {
  const int32_t nz = st->nnz_y;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nz; k += gridDim.x * blockDim.x) {
    const int32_t i = z_idx[k];
    atomicOr(&decided[i >> 5], 1u << (i & 31));
  }
}

// x restricted to the vertices still undecided, written to (t_idx, t_val)
__global__ void k_mis_compact(const int32_t* __restrict__ x_idx, const uint32_t* __restrict__ x_val,
                              const uint32_t* __restrict__ decided, int32_t* __restrict__ t_idx,
                              uint32_t* __restrict__ t_val, int32_t* __restrict__ cnt) {
  const int32_t nc = cnt[0];
  const int lane = threadIdx.x & 31;
  for (int32_t k0 = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; k0 < nc;
       k0 += gridDim.x * blockDim.x) {
    const int32_t k = k0 + lane;
    int32_t v = 0;
    uint32_t p = 0u;
    bool keep = false;
    if (k < nc) {
      v = x_idx[k];
      p = x_val[k];
      keep = !((decided[v >> 5] >> (v & 31)) & 1u);
    }
    const int32_t pos = warp_append(keep, &cnt[2]);
    if (keep) {
      t_idx[pos] = v;
      t_val[pos] = p;
    }
  }
}

__global__ void k_mis_copy(const int32_t* __restrict__ t_idx, const uint32_t* __restrict__ t_val,
                           int32_t* __restrict__ x_idx, uint32_t* __restrict__ x_val,
                           const int32_t* __restrict__ cnt) {
  const int32_t nk = cnt[2];
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nk; k += gridDim.x * blockDim.x) {
    x_idx[k] = t_idx[k];
    x_val[k] = t_val[k];
  }
}

__global__ void k_mis_continue(cudaGraphConditionalHandle cond, DevState* st, int32_t* cnt, int32_t n) {
  if (threadIdx.x == 0) {
    cnt[0] = cnt[2];
    cnt[1] = 0;
    cnt[2] = 0;
    st->level += 1;
    cudaGraphSetConditional(cond, (cnt[0] > 0 && st->level <= n) ? 1u : 0u);
  }
}

}  // namespace

static int mis_round_launches(spmspv_handle* h, const Sched& sc, cudaGraphConditionalHandle cond,
                              cudaStream_t s) {
  const int g = h->sm_count * 4;
  int rc = graph_spmspv(h, kMinSelect2nd, sc, h->mis_x_idx, h->mis_x_val, &h->mis_cnt[0],
                        h->mis_decided, h->mis_y_idx, h->mis_y_val, s);
  if (rc != SPMSPV_OK) return rc;
  k_mis_scatter<<<g, 256, 0, s>>>(h->ws.st, h->mis_y_idx, h->mis_y_val, h->mis_ymin);
  k_mis_join<<<g, 256, 0, s>>>(h->ws.st, h->mis_x_idx, h->mis_x_val, h->mis_ymin, h->mis_decided,
                               h->mis_j_idx, h->mis_cnt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "mis join");
  if ((rc = graph_spmspv(h, kOrAnd, sc, h->mis_j_idx, nullptr, &h->mis_cnt[1], h->mis_decided,
                         h->mis_y_idx, nullptr, s)) != SPMSPV_OK)
    return rc;
  k_mis_remove<<<g, 256, 0, s>>>(h->ws.st, h->mis_y_idx, h->mis_decided);
  k_mis_compact<<<g, 256, 0, s>>>(h->mis_x_idx, h->mis_x_val, h->mis_decided, h->mis_y_idx,
                                  h->mis_y_val, h->mis_cnt);
  k_mis_copy<<<g, 256, 0, s>>>(h->mis_y_idx, h->mis_y_val, h->mis_x_idx, h->mis_x_val, h->mis_cnt);
  k_mis_continue<<<1, 32, 0, s>>>(cond, h->ws.st, h->mis_cnt, h->A.n);
  return (e = cudaGetLastError()) == cudaSuccess ? SPMSPV_OK : cuda_fail(e, "mis round");
}

void release_mis(spmspv_handle* h) {
  for (int i = 0; i < SPMSPV_NUM_SCHEDULES / 2; ++i) {
    if (h->mis_graph[i]) cudaGraphExecDestroy((cudaGraphExec_t)h->mis_graph[i]);
    h->mis_graph[i] = nullptr;
  }
  cudaFree(h->mis_x_idx);
  cudaFree(h->mis_x_val);
  cudaFree(h->mis_y_idx);
  cudaFree(h->mis_y_val);
  cudaFree(h->mis_j_idx);
  cudaFree(h->mis_ymin);
  cudaFree(h->mis_decided);
  cudaFree(h->mis_cnt);
  h->mis_x_idx = nullptr;
  h->mis_x_val = nullptr;
  h->mis_y_idx = nullptr;
  h->mis_y_val = nullptr;
  h->mis_j_idx = nullptr;
  h->mis_ymin = nullptr;
  h->mis_decided = nullptr;
  h->mis_cnt = nullptr;
}

}  // namespace spmspv

using namespace spmspv;

extern "C" int spmspv_mis(spmspv_handle* h, const int32_t* prio, int32_t* in_set, int32_t* d_nrounds,
                          uint32_t opts, spmspv_stream_t stream) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (h->A.m != h->A.n) return fail(SPMSPV_ERR_ARG, "an independent set needs a square matrix");
  if (!(h->flags & SPMSPV_CSC_PATTERN_SYMMETRIC))
    return fail(SPMSPV_ERR_ARG, "an independent set needs a pattern-symmetric (undirected) matrix");
  if (!prio || !in_set) return fail(SPMSPV_ERR_ARG, "prio or in_set is NULL");
  if (opts & SPMSPV_SCHED_AUTO) return fail(SPMSPV_ERR_UNSUPPORTED, "the independent set runs a fixed push schedule");
  int sched = h->default_sched;
  if (opts & SPMSPV_SCHED_FORCE) sched = (int)SPMSPV_SCHED_ID(opts);
  if (sched < 0 || sched >= SPMSPV_NUM_SCHEDULES / 2)
    return fail(SPMSPV_ERR_ARG, "the independent set takes a push schedule (0..5)");
  const size_t n = (size_t)h->A.n;
  const size_t nw = (n + 31) / 32;
  if (!h->mis_x_idx) {
    cudaError_t e = cudaMalloc(&h->mis_x_idx, sizeof(int32_t) * std::max<size_t>(n, 1));
    if (e == cudaSuccess) e = cudaMalloc(&h->mis_x_val, sizeof(uint32_t) * std::max<size_t>(n, 1));
    if (e == cudaSuccess) e = cudaMalloc(&h->mis_y_idx, sizeof(int32_t) * std::max<size_t>(n, 1));
    if (e == cudaSuccess) e = cudaMalloc(&h->mis_y_val, sizeof(uint32_t) * std::max<size_t>(n, 1));
    if (e == cudaSuccess) e = cudaMalloc(&h->mis_j_idx, sizeof(int32_t) * std::max<size_t>(n, 1));
    if (e == cudaSuccess) e = cudaMalloc(&h->mis_ymin, sizeof(int32_t) * std::max<size_t>(n, 1));
    if (e == cudaSuccess) e = cudaMalloc(&h->mis_decided, sizeof(uint32_t) * std::max<size_t>(nw, 1));
    if (e == cudaSuccess) e = cudaMalloc(&h->mis_cnt, sizeof(int32_t) * 4);
    if (e != cudaSuccess) {
      release_mis(h);
      cudaGetLastError();
      return fail(SPMSPV_ERR_OOM, "independent-set buffers: %s", cudaGetErrorString(e));
    }
  }
  if (!h->mis_graph[sched]) {
    cudaGraphExec_t exec = nullptr;
    const Sched sc = decode_schedule(h, sched);
    rc = build_while_graph(h, [&](cudaGraphConditionalHandle c, cudaStream_t cs) {
      return mis_round_launches(h, sc, c, cs);
    }, &exec);
    if (rc != SPMSPV_OK) return rc;
    h->mis_graph[sched] = exec;
  }
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  h->last_empty = 0;
  const int grid = std::max(1, std::min(h->sm_count * 8, (h->A.n + 255) / 256));
  k_mis_init<<<grid, 256, 0, s>>>(h->A.n, prio, in_set, h->mis_x_idx, h->mis_x_val, h->mis_ymin,
                                  h->mis_decided, h->mis_cnt, h->ws.st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "mis init");
  if ((e = cudaGraphLaunch((cudaGraphExec_t)h->mis_graph[sched], s)) != cudaSuccess)
    return cuda_fail(e, "mis graph launch");
  if (d_nrounds) {
    e = cudaMemcpyAsync(d_nrounds, &h->ws.st->level, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "mis round count");
  }
  return SPMSPV_OK;
}
