// Breadth-first search as repeated masked (min, select2nd) SpMSpV (Sec. IV-D):
// frontier x = {(j, j)}, y = A (min.select2nd) x on the unvisited rows, every
// (i, p) in y gets level L and parent p, joins the visited mask and forms the
// next frontier; stop at an empty y.
//
// The whole level loop runs on the device: a CUDA graph with a conditional
// WHILE node whose body is one level (work scan -> [selector] -> push kernels
// | pull kernels -> condition kernel).  The condition kernel keeps the loop
// going while the last y was non-empty, so a search of thousands of levels
// never returns to the host.  One graph is built per handle and schedule mode
// on first use and reused; the per-search arguments (source, output arrays)
// reach the kernels through the device state.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "handle.cuh"
#include "spmspv_internal.cuh"

namespace spmspv {

cudaError_t launch_pull(const spmspv_handle* h, int sem, bool bfs, const int32_t* x_idx,
                        const uint32_t* x_val, int f, const int32_t* f_dev, const uint32_t* mask,
                        int mask_comp, int early_exit, int32_t* y_idx, uint32_t* y_val,
                        int32_t y_cap, int32_t* d_nnz_y, uint32_t* visited, int only_pull,
                        cudaStream_t s);
cudaError_t launch_pull_rows_bfs(const spmspv_handle* h, int early_exit, int only_pull, cudaStream_t s,
                                 cudaGraphConditionalHandle cond);
int pull_available(const spmspv_handle* h, int sem);

namespace {

// Start of a search: every vertex unreached, the source at level 0.
// keep_fb: the search may run pull levels, which read the last level's
// frontier bitmap (kept only then: the push levels skip its upkeep otherwise).
__global__ void k_bfs_init(int32_t n, int32_t src, int32_t* __restrict__ level,
                           int32_t* __restrict__ parent, uint32_t* __restrict__ visited,
                           uint32_t* __restrict__ fb, int32_t* __restrict__ front, DevState* st,
                           int keep_fb) {
  const int32_t words = (n + 31) / 32;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    level[i] = i == src ? 0 : -1;
    parent[i] = i == src ? src : -1;
    if (i < words) {
      const uint32_t w = (i == (src >> 5)) ? (1u << (src & 31)) : 0u;
      visited[i] = w;
      fb[i] = w;       // level 0's frontier, read by a pull at level 1
      fb[words + i] = 0u;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    front[0] = src;
    st->nnz_y = 1;
    st->level = 0;
    st->nvisited = 1;
    st->bfs_level = level;
    st->bfs_parent = parent;
    st->bfs_fb = keep_fb ? fb : nullptr;
    st->bfs_front = front;
    st->fused_count = 0u;
    st->fused_gen = 0u;
    st->fused_w[3] = 0;
    st->fused_fc[3] = 0;
    st->fused_md[3] = 0;
    st->edges_seen = 0;
    st->dir = 0;  // the rule starts in the push direction
  }
}

}  // namespace

// device_sched: the work scan picks the schedule, so K2 must not be the
// variant compiled for one work quantum.
static int bfs_push_launches(spmspv_handle* h, const Sched& sc, int lwb, cudaStream_t s, int only_push,
                             bool device_sched, cudaGraphConditionalHandle cond) {
  const size_t k3_smem = k3_smem_bytes(lwb);
  const int nb_max = (int)(((int64_t)h->A.m + (1 << h->lwb_lo) - 1) >> h->lwb_lo);
  const int k3_grid = std::max(1, std::min(nb_max, h->sm_count * h->k3_bps[lwb - h->lwb_lo]));
  cudaError_t e = launch_k2(kMinSelect2nd, h->A, h->ws, h->lwb_lo, h->nb_fine, h->bfs_visited, 1,
                            h->k2_grid, h->k2_smem, s, only_push, device_sched ? 0 : sc.q, BFS_DIRECT_MAX);
  if (e != cudaSuccess) return cuda_fail(e, "bfs expand/scatter");
  e = launch_k3(kMinSelect2nd, true, h->A, h->ws, h->lwb_lo, h->nb_fine, h->bfs_front, nullptr,
                h->A.n, nullptr, h->bfs_visited, k3_grid, k3_smem, s, only_push, BFS_DIRECT_MAX, 1, cond);
  return e == cudaSuccess ? SPMSPV_OK : cuda_fail(e, "bfs merge");
}

static int bfs_pull_launches(spmspv_handle* h, int only_pull, cudaStream_t s, cudaGraphConditionalHandle cond) {
  cudaError_t e = launch_pull_rows_bfs(h, h->rows_sorted, only_pull, s, cond);
  return e == cudaSuccess ? SPMSPV_OK : cuda_fail(e, "bfs pull");
}

// One BFS level on `s` (captured into the loop body).  A fixed schedule
// launches its direction's kernels; the learned schedule launches the work
// scan, whose last CTA runs the selector, then the push and the pull kernels,
// of which the ones not chosen return at once.
static int bfs_level_launches(spmspv_handle* h, int sched, cudaGraphConditionalHandle cond,
                              cudaStream_t s) {
  const bool autos = sched < 0;  // -1: the learned selector, -2: the direction-optimizing rule
  const bool can_pull = pull_available(h, kMinSelect2nd) != 0;
  Sched sc = decode_schedule(h, autos ? h->default_sched : sched);
  if (!can_pull && sc.dir == 1) {
    sc.dir = 0;
    sc.id %= 6;
  }
  cudaError_t e;
  int rc = SPMSPV_OK;
  if (!autos) {
    if ((e = launch_k1_bfs(h->A, h->ws, h->nb_fine, h->bfs_front, &h->ws.st->nnz_y, h->k1_grid_dev, &sc,
                           s, nullptr)) != cudaSuccess)
      return cuda_fail(e, "bfs work scan");
    rc = sc.dir == 0 ? bfs_push_launches(h, sc, sc.lwb, s, 0, false, cond) : bfs_pull_launches(h, 0, s, cond);
  } else {
    // the work scan's last CTA runs the selector and sets the direction; the
    // push kernels and the pull kernel both follow and the one not chosen
    // returns at once (no conditional nodes); the visited count stands in
    // for a pass over the visited bitmap
    SelArgs sa{};
    sa.w = sched == -2 ? nullptr : h->sel_w;
    sa.rule = sched == -2 ? 1 : 0;
    sa.allow_pull = can_pull;
    sa.bfs = 1;
    sa.lwb_lo = h->lwb_lo;
    sa.direct_max = BFS_DIRECT_MAX;
    if ((e = launch_k1_bfs(h->A, h->ws, h->nb_fine, h->bfs_front, &h->ws.st->nnz_y, h->k1_grid_dev,
                           nullptr, s, nullptr, &sa)) != cudaSuccess)
      return cuda_fail(e, "bfs work scan");
    rc = bfs_push_launches(h, sc, h->lwb_lo + 2, s, can_pull ? 1 : 0, true, cond);
    if (rc == SPMSPV_OK && can_pull) rc = bfs_pull_launches(h, 1, s, cond);
  }
  // the kernel that closes the level (K3, or the pull kernel) sets the loop's
  // condition: no launch of its own
  return rc;
}

// Graph with one WHILE node whose body is one level.
static int build_bfs_graph(spmspv_handle* h, int sched, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
  int rc = SPMSPV_OK;
  do {
    cudaGraphConditionalHandle cond;
    if ((e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess) {
      rc = cuda_fail(e, "cudaGraphConditionalHandleCreate");
      break;
    }
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np)) != cudaSuccess) {
      rc = cuda_fail(e, "add while node");
      break;
    }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) {
      rc = cuda_fail(e, "capture stream");
      break;
    }
    if ((e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
      rc = cuda_fail(e, "begin capture");
      break;
    }
    void* saved_prof = h->prof;
    h->prof = nullptr;  // no profiling events inside the graph
    rc = bfs_level_launches(h, sched, cond, cs);
    h->prof = saved_prof;
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(cs, &captured);
    if (rc != SPMSPV_OK) break;
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "end capture");
      break;
    }
    if ((e = cudaGraphInstantiate(&exec, g, 0)) != cudaSuccess) {
      rc = cuda_fail(e, "instantiate bfs graph");
      break;
    }
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

int ensure_bfs_buffers(spmspv_handle* h) {
  if (h->bfs_front) return SPMSPV_OK;
  const size_t n = (size_t)h->A.n;
  // the persistent kernel of the learned schedule runs on CSC handles
  const int fg = h->A.jc ? 0 : fused_bfs_grid(h);
  cudaError_t e = cudaMalloc(&h->bfs_front, sizeof(int32_t) * n);
  if (e == cudaSuccess) e = cudaMalloc(&h->bfs_visited, sizeof(uint32_t) * ((n + 31) / 32 + 1));
  if (e == cudaSuccess) e = cudaMalloc(&h->bfs_fb, sizeof(uint32_t) * 2 * ((n + 31) / 32));
  if (e == cudaSuccess && fg > 0) e = cudaMalloc(&h->bfs_front2, sizeof(int32_t) * n);
  if (e == cudaSuccess && fg > 0) e = cudaMalloc(&h->bfs_slice, sizeof(int32_t) * 3 * (size_t)fg);
  if (e != cudaSuccess) {
    cudaFree(h->bfs_front);
    cudaFree(h->bfs_visited);
    cudaFree(h->bfs_fb);
    cudaFree(h->bfs_front2);
    cudaFree(h->bfs_slice);
    h->bfs_front = nullptr;
    h->bfs_visited = nullptr;
    h->bfs_fb = nullptr;
    h->bfs_front2 = nullptr;
    h->bfs_slice = nullptr;
    cudaGetLastError();
    return fail(SPMSPV_ERR_OOM, "BFS buffers: %s", cudaGetErrorString(e));
  }
  h->fused_grid = fg;
  return SPMSPV_OK;
}

void release_bfs_graphs(spmspv_handle* h) {
  for (int i = 0; i < SPMSPV_NUM_SCHEDULES + 2; ++i) {
    if (h->bfs_graph[i]) cudaGraphExecDestroy((cudaGraphExec_t)h->bfs_graph[i]);
    h->bfs_graph[i] = nullptr;
  }
}

}  // namespace spmspv

using namespace spmspv;

extern "C" int spmspv_bfs(spmspv_handle* h, int32_t src, int32_t* level, int32_t* parent,
                          int32_t* d_nlevels, uint32_t opts, spmspv_stream_t stream) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (h->A.m != h->A.n) return fail(SPMSPV_ERR_ARG, "BFS needs a square matrix");
  if (src < 0 || src >= h->A.n) return fail(SPMSPV_ERR_ARG, "src = %d outside [0, n)", src);
  if (!level || !parent) return fail(SPMSPV_ERR_ARG, "level or parent is NULL");
  if ((opts & SPMSPV_SCHED_FORCE) && SPMSPV_SCHED_ID(opts) >= SPMSPV_NUM_SCHEDULES)
    return fail(SPMSPV_ERR_ARG, "schedule id out of range");
  int sched = h->default_sched;
  if (opts & SPMSPV_SCHED_FORCE) sched = (int)SPMSPV_SCHED_ID(opts);
  if ((opts & SPMSPV_SCHED_AUTO) && (opts & SPMSPV_SCHED_RULE))
    return fail(SPMSPV_ERR_ARG, "SPMSPV_SCHED_AUTO and SPMSPV_SCHED_RULE exclude each other");
  if (opts & SPMSPV_SCHED_AUTO) {
    if (!h->sel_ready) return fail(SPMSPV_ERR_STATE, "no selector weights loaded or trained");
    sched = -1;
  }
  if (opts & SPMSPV_SCHED_RULE) sched = -2;
  if ((rc = ensure_bfs_buffers(h)) != SPMSPV_OK) return rc;
  const int slot = sched == -1 ? SPMSPV_NUM_SCHEDULES : sched == -2 ? SPMSPV_NUM_SCHEDULES + 1 : sched;
  if (!h->bfs_graph[slot]) {
    cudaGraphExec_t exec = nullptr;
    if ((rc = build_bfs_graph(h, sched, &exec)) != SPMSPV_OK) return rc;
    h->bfs_graph[slot] = exec;
  }
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  h->last_empty = 0;
  const int grid = std::max(1, std::min(h->sm_count * 8, (h->A.n + 255) / 256));
  const bool pulls = pull_available(h, kMinSelect2nd) && (sched < 0 || sched >= SPMSPV_NUM_SCHEDULES / 2);
  k_bfs_init<<<grid, 256, 0, s>>>(h->A.n, src, level, parent, h->bfs_visited, h->bfs_fb, h->bfs_front,
                                  h->ws.st, pulls ? 1 : 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "bfs init");
  // the adaptive schedules (learned, rule): the first levels, as long as
  // they are small push levels, in one persistent launch (on a high-diameter
  // graph usually the whole search); it leaves the state of the first level
  // it does not run to the graph's loop of plain kernels
  if (sched < 0 && h->fused_grid > 0 && (e = launch_bfs_fused(h, h->fused_grid, s)) != cudaSuccess)
    return cuda_fail(e, "bfs persistent levels");
  if ((e = cudaGraphLaunch((cudaGraphExec_t)h->bfs_graph[slot], s)) != cudaSuccess)
    return cuda_fail(e, "bfs graph launch");
  if (d_nlevels) {
    e = cudaMemcpyAsync(d_nlevels, &h->ws.st->level, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "bfs level count");
  }
  return SPMSPV_OK;
}
