// Maximum-cardinality matching of the bipartite graph between the rows and
// the columns of A by phases of multi-source alternating BFS, one masked
// (min.select2nd) SpMSpV per BFS level.  Sec. I names bipartite graph
// matching among the graph algorithms whose workhorse is SpMSpV; the paper
// gives no algorithm, so the phases below are this library's reading.
//
//   phase:  roots = free columns;  x = {(j, j) : j a root};  visited rows = {}
//     level:  y = A (min.select2nd) x, rows masked to the unvisited
//                 y(i) = the smallest frontier column next to row i (its parent)
//             for (i, p) in y:  visit i;  r = root(p)
//               i free:     i ends an augmenting path of tree r (the first such
//                           row per tree is kept)
//               i matched:  its mate column joins tree r and the next frontier,
//                           unless tree r already has its path
//     until the frontier is empty;
//     then flip every kept path (rows and columns along it swap mates).
//   until a phase finds no path.
//
// Trees of a phase share no vertex (each row is visited once, and a matched
// column is reached only through its mate), so the kept paths are disjoint and
// each flip adds one edge to the matching.  A phase that finds no path has
// searched every alternating path from every free column, so the matching is
// then maximum (Berge).  Levels and phases run in one CUDA graph: a WHILE node
// whose body is one level plus the end-of-phase kernels, which return at once
// on the levels where the phase goes on.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "device_util.cuh"
#include "handle.cuh"
#include "spmspv_internal.cuh"

namespace spmspv {
namespace {

// cnt[0] frontier length, cnt[1] next frontier, cnt[2] paths of this phase,
// cnt[3] the next phase's frontier, cnt[4] phases with a path, cnt[5] level in
// the phase, cnt[6] cardinality
constexpr int kCnt = 8;

__global__ void k_mcm_init(int32_t m, int32_t n, int32_t* __restrict__ mate_r, int32_t* __restrict__ mate_c,
                           int32_t* __restrict__ x_idx, int32_t* __restrict__ root_c,
                           int32_t* __restrict__ leaf, uint32_t* __restrict__ visited,
                           int32_t* __restrict__ cnt, DevState* st) {
  const int32_t mw = (m + 31) >> 5;
  const int32_t top = m > n ? m : n;
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < top; v += gridDim.x * blockDim.x) {
    if (v < m) mate_r[v] = -1;
    if (v < mw) visited[v] = 0u;
    if (v < n) {
      mate_c[v] = -1;
      x_idx[v] = v;
      root_c[v] = v;
      leaf[v] = -1;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x < kCnt) cnt[threadIdx.x] = threadIdx.x == 0 ? n : 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->level = 0;
    st->mcm_mate_r = mate_r;
    st->mcm_mate_c = mate_c;
  }
}

// One level's y: visit the rows, keep one free row per tree, grow the trees
// without a path through the mates of the matched rows.
__global__ void k_mcm_level(const DevState* __restrict__ st, const int32_t* __restrict__ y_idx,
                            const uint32_t* __restrict__ y_val, int32_t* __restrict__ parent_r,
                            int32_t* __restrict__ root_c, int32_t* leaf, uint32_t* __restrict__ visited,
                            int32_t* __restrict__ x2_idx, int32_t* __restrict__ cnt) {
  const int32_t* const mate_r = st->mcm_mate_r;
  const int32_t ny = st->nnz_y;
  const int lane = threadIdx.x & 31;
  // grid-stride in whole warps so that every lane of a warp takes part in the ballot
  for (int32_t k0 = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; k0 < ny;
       k0 += gridDim.x * blockDim.x) {
    const int32_t k = k0 + lane;
    int32_t mi = -1, r = 0;
    bool grow = false;
    if (k < ny) {
      const int32_t i = y_idx[k];
      const int32_t p = (int32_t)y_val[k];
      atomicOr(&visited[i >> 5], 1u << (i & 31));
      parent_r[i] = p;
      r = root_c[p];
      mi = mate_r[i];
      if (mi < 0) {
        if (atomicCAS(&leaf[r], -1, i) == -1) atomicAdd(&cnt[2], 1);
      } else {
        // a tree that has its path stops growing (a stale read only costs work)
        grow = *((volatile const int32_t*)&leaf[r]) < 0;
      }
    }
    const int32_t pos = warp_append(grow, &cnt[1]);
    if (grow) {
      root_c[mi] = r;
      x2_idx[pos] = mi;
    }
  }
}

__global__ void k_mcm_copy(const int32_t* __restrict__ x2_idx, int32_t* __restrict__ x_idx,
                           const int32_t* __restrict__ cnt) {
  const int32_t nk = cnt[1];
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < nk; k += gridDim.x * blockDim.x)
    x_idx[k] = x2_idx[k];
}

// End of a phase with paths: flip each kept path, walking from its free row
// to its root through the row parents and the old mates of the columns.
__global__ void k_mcm_augment(DevState* st, int32_t m, int32_t n, const int32_t* __restrict__ parent_r,
                              int32_t* __restrict__ leaf, const int32_t* __restrict__ cnt) {
  if (cnt[1] != 0 || cnt[2] == 0) return;
  int32_t* const mate_r = st->mcm_mate_r;
  int32_t* const mate_c = st->mcm_mate_c;
  for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    int32_t i = leaf[r];
    if (i < 0) continue;
    leaf[r] = -1;
    bool done = false;
    // a path has at most one row per visited row: m steps bound the walk
    for (int32_t step = 0; step <= m && i >= 0; ++step) {
      const int32_t j = parent_r[i];
      if (j < 0 || j >= n) break;  // not a parent set in this phase: reported below
      const int32_t old = mate_c[j];
      mate_c[j] = i;
      mate_r[i] = j;
      if (j == r) {
        done = true;
        break;
      }
      i = old;
    }
    if (!done) atomicOr(&st->status, ST_BOUND);
  }
}

// Start of the next phase: clear the visited rows, the free non-empty
// columns become the roots and the frontier.
__global__ void k_mcm_new_phase(int32_t m, int32_t n, Matrix A, const DevState* __restrict__ st, int32_t* __restrict__ x_idx,
                                int32_t* __restrict__ root_c, uint32_t* __restrict__ visited,
                                int32_t* __restrict__ cnt) {
  if (cnt[1] != 0 || cnt[2] == 0) return;
  const int32_t* const mate_c = st->mcm_mate_c;
  const int32_t mw = (m + 31) >> 5;
  for (int32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < mw; w += gridDim.x * blockDim.x)
    visited[w] = 0u;
  const int lane = threadIdx.x & 31;
  for (int32_t j0 = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; j0 < n; j0 += gridDim.x * blockDim.x) {
    const int32_t j = j0 + lane;
    bool root = j < n && mate_c[j] < 0;
    if (root) {
      int32_t c0, c1;
      col_range(A.colptr, A.jc, A.aux, A.aux_shift, j, c0, c1);
      root = c1 > c0;
    }
    const int32_t pos = warp_append(root, &cnt[3]);
    if (root) {
      root_c[j] = j;
      x_idx[pos] = j;
    }
  }
}

__global__ void k_mcm_continue(cudaGraphConditionalHandle cond, DevState* st, int32_t* cnt, int32_t m,
                               int32_t n) {
  if (threadIdx.x != 0) return;
  const int32_t nxt = cnt[1], paths = cnt[2];
  bool go;
  if (nxt > 0) {  // the phase goes on
    cnt[0] = nxt;
    cnt[5] += 1;
    go = true;
  } else if (paths > 0) {  // paths flipped: next phase
    cnt[6] += paths;
    cnt[4] += 1;
    cnt[0] = cnt[3];
    cnt[2] = 0;
    cnt[5] = 0;
    go = cnt[3] > 0;
  } else {  // no path left: the matching is maximum
    go = false;
  }
  cnt[1] = 0;
  cnt[3] = 0;
  // every level visits a new row and every phase adds a matched pair
  if (cnt[5] > m || cnt[4] > (m < n ? m : n)) {
    atomicOr(&st->status, ST_BOUND);
    go = false;
  }
  st->level = cnt[4];
  cudaGraphSetConditional(cond, go ? 1u : 0u);
}

}  // namespace

static int mcm_level_launches(spmspv_handle* h, const Sched& sc, cudaGraphConditionalHandle cond,
                              cudaStream_t s) {
  const int g = h->sm_count * 4;
  int rc = graph_spmspv(h, kMinSelect2nd, sc, h->mcm_x_idx, nullptr, &h->mcm_cnt[0], h->mcm_visited,
                        h->mcm_y_idx, h->mcm_y_val, s);
  if (rc != SPMSPV_OK) return rc;
  k_mcm_level<<<g, 256, 0, s>>>(h->ws.st, h->mcm_y_idx, h->mcm_y_val, h->mcm_parent_r, h->mcm_root_c,
                                h->mcm_leaf, h->mcm_visited, h->mcm_x2_idx, h->mcm_cnt);
  k_mcm_copy<<<g, 256, 0, s>>>(h->mcm_x2_idx, h->mcm_x_idx, h->mcm_cnt);
  k_mcm_augment<<<g, 256, 0, s>>>(h->ws.st, h->A.m, h->A.n, h->mcm_parent_r, h->mcm_leaf, h->mcm_cnt);
  k_mcm_new_phase<<<g, 256, 0, s>>>(h->A.m, h->A.n, h->A, h->ws.st, h->mcm_x_idx, h->mcm_root_c,
                                    h->mcm_visited, h->mcm_cnt);
  k_mcm_continue<<<1, 32, 0, s>>>(cond, h->ws.st, h->mcm_cnt, h->A.m, h->A.n);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPMSPV_OK : cuda_fail(e, "matching level");
}

void release_mcm(spmspv_handle* h) {
  for (int i = 0; i < SPMSPV_NUM_SCHEDULES / 2; ++i) {
    if (h->mcm_graph[i]) cudaGraphExecDestroy((cudaGraphExec_t)h->mcm_graph[i]);
    h->mcm_graph[i] = nullptr;
  }
  cudaFree(h->mcm_x_idx);
  cudaFree(h->mcm_x2_idx);
  cudaFree(h->mcm_y_idx);
  cudaFree(h->mcm_y_val);
  cudaFree(h->mcm_parent_r);
  cudaFree(h->mcm_root_c);
  cudaFree(h->mcm_leaf);
  cudaFree(h->mcm_visited);
  cudaFree(h->mcm_cnt);
  h->mcm_x_idx = nullptr;
  h->mcm_x2_idx = nullptr;
  h->mcm_y_idx = nullptr;
  h->mcm_y_val = nullptr;
  h->mcm_parent_r = nullptr;
  h->mcm_root_c = nullptr;
  h->mcm_leaf = nullptr;
  h->mcm_visited = nullptr;
  h->mcm_cnt = nullptr;
}

}  // namespace spmspv

using namespace spmspv;

extern "C" int spmspv_mcm(spmspv_handle* h, int32_t* mate_r, int32_t* mate_c, int32_t* d_card,
                          int32_t* d_nphases, uint32_t opts, spmspv_stream_t stream) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!mate_r || !mate_c) return fail(SPMSPV_ERR_ARG, "mate_r or mate_c is NULL");
  if (opts & SPMSPV_SCHED_AUTO) return fail(SPMSPV_ERR_UNSUPPORTED, "the matching runs a fixed push schedule");
  int sched = h->default_sched;
  if (opts & SPMSPV_SCHED_FORCE) sched = (int)SPMSPV_SCHED_ID(opts);
  if (sched < 0 || sched >= SPMSPV_NUM_SCHEDULES / 2)
    return fail(SPMSPV_ERR_ARG, "the matching takes a push schedule (0..5)");
  const size_t m = (size_t)h->A.m, n = (size_t)h->A.n;
  const size_t mw = (m + 31) / 32;
  if (!h->mcm_x_idx) {
    cudaError_t e = cudaMalloc(&h->mcm_x_idx, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&h->mcm_x2_idx, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&h->mcm_y_idx, sizeof(int32_t) * m);
    if (e == cudaSuccess) e = cudaMalloc(&h->mcm_y_val, sizeof(uint32_t) * m);
    if (e == cudaSuccess) e = cudaMalloc(&h->mcm_parent_r, sizeof(int32_t) * m);
    if (e == cudaSuccess) e = cudaMalloc(&h->mcm_root_c, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&h->mcm_leaf, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&h->mcm_visited, sizeof(uint32_t) * mw);
    if (e == cudaSuccess) e = cudaMalloc(&h->mcm_cnt, sizeof(int32_t) * kCnt);
    if (e != cudaSuccess) {
      release_mcm(h);
      cudaGetLastError();
      return fail(SPMSPV_ERR_OOM, "matching buffers: %s", cudaGetErrorString(e));
    }
  }
  if (!h->mcm_graph[sched]) {
    cudaGraphExec_t exec = nullptr;
    const Sched sc = decode_schedule(h, sched);
    rc = build_while_graph(h, [&](cudaGraphConditionalHandle c, cudaStream_t cs) {
      return mcm_level_launches(h, sc, c, cs);
    }, &exec);
    if (rc != SPMSPV_OK) return rc;
    h->mcm_graph[sched] = exec;
  }
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  h->last_empty = 0;
  const int32_t top = std::max(h->A.m, h->A.n);
  const int grid = std::max(1, std::min(h->sm_count * 8, (top + 255) / 256));
  k_mcm_init<<<grid, 256, 0, s>>>(h->A.m, h->A.n, mate_r, mate_c, h->mcm_x_idx, h->mcm_root_c, h->mcm_leaf,
                                  h->mcm_visited, h->mcm_cnt, h->ws.st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "matching init");
  if ((e = cudaGraphLaunch((cudaGraphExec_t)h->mcm_graph[sched], s)) != cudaSuccess)
    return cuda_fail(e, "matching graph launch");
  if (d_card) {
    e = cudaMemcpyAsync(d_card, &h->mcm_cnt[6], sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "matching cardinality");
  }
  if (d_nphases) {
    e = cudaMemcpyAsync(d_nphases, &h->mcm_cnt[4], sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "matching phase count");
  }
  return SPMSPV_OK;
}
