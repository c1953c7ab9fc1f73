// Batched SpMSpV, the lanes form: B independent products y_b <- A (+).(x) x_b
// in one graph launch (the persistent one-launch form is batched_k6.cu), and
// the multi-source BFS and ACL drivers, whose level / push steps run on
// either form (this file holds their per-source kernels: the persistent
// form's level update, learned push/pull decision and batched pull).  The
// paper runs one product per call; repeated small calls are where it notes
// most time goes to overhead (Sec. I, Sec. III-A), so the batch is run as L
// concurrent "lanes": each lane is a device-side WHILE
// loop (a conditional graph node) that pops the next frontier from a queue
// shared by the lanes and runs the same three kernels (work scan ->
// expand/scatter -> bucket merge) on it with its own workspace.  No frontier
// waits for the host, the lanes keep the GPU busy while small frontiers leave
// most of it idle, and every frontier gets exactly the result of a single
// spmspv_run call with the same schedule.
//
// The graph is built once per (semiring, lanes, schedule, mode) and reused;
// the per-call arrays reach the kernels through a device batch descriptor
// and one job descriptor per lane.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "handle.cuh"
#include "selector_dev.cuh"
#include "spmspv_internal.cuh"

namespace spmspv {

struct BatchDesc {
  int32_t B;
  int32_t head;  // queue head (atomic)
  int32_t lvl;   // BFS mode: level being discovered
  int32_t dummy_nnz;
  const int32_t* x_off;
  const int32_t* x_cnt;
  const int32_t* x_idx;
  const uint32_t* x_val;
  const uint32_t* masks;
  int64_t mask_stride;
  const int32_t* y_off;
  const int32_t* y_cap;
  int32_t* y_idx;
  uint32_t* y_val;
  int32_t* d_nnz_y;
  int32_t* level;   // BFS mode: [B][n]
  int32_t* parent;  // BFS mode: [B][n]
  int64_t vstride;  // n
  uint32_t* fb;     // learned BFS: [B][2][ceil(n/32)] frontier bitmaps
  int64_t fb_stride;
  const int32_t* nvis;  // learned BFS: [B] vertices reached per source
};

struct BatchState {
  int lanes;
  spmspv_handle* sub[MAX_LANES];  // one workspace per lane
  Job* jobs;                      // [MAX_LANES] device
  BatchDesc* desc;                // device
  // [semiring][schedule, or SPMSPV_NUM_SCHEDULES for the learned BFS][bfs][lanes]
  cudaGraphExec_t graphs[3][SPMSPV_NUM_SCHEDULES + 1][2][MAX_LANES + 1];
};

namespace {

__global__ void k_batch_start(BatchDesc* d, BatchDesc v) {
  if (threadIdx.x == 0) {
    v.head = 0;
    v.dummy_nnz = 0;
    v.lvl = d->lvl;
    *d = v;
  }
}

__global__ void k_batch_set_level(BatchDesc* d, int32_t lvl) {
  if (threadIdx.x == 0) d->lvl = lvl;
}

// Lane step 1: take the next frontier (or an empty job when none is left).
__global__ void k_batch_pop(BatchDesc* d, Job* job) {
  if (threadIdx.x != 0) return;
  const int32_t t = atomicAdd(&d->head, 1);
  Job j;
  memset(&j, 0, sizeof(j));
  j.b = -1;
  j.d_nnz_y = &d->dummy_nnz;
  j.x_idx = d->x_idx;
  if (t < d->B) {
    const int32_t b = t;
    const int32_t xo = d->x_off[b];
    j.b = b;
    j.f = d->x_cnt[b];
    j.x_idx = d->x_idx + xo;
    j.x_val = d->x_val ? d->x_val + xo : nullptr;
    j.mask = d->masks ? d->masks + (int64_t)b * d->mask_stride : nullptr;
    j.y_idx = d->y_idx + d->y_off[b];
    j.y_val = d->y_val ? d->y_val + d->y_off[b] : nullptr;
    j.y_cap = d->y_cap[b];
    j.d_nnz_y = d->d_nnz_y + b;
    if (d->level) {
      j.level = d->level + (int64_t)b * d->vstride;
      j.parent = d->parent + (int64_t)b * d->vstride;
      j.visited = const_cast<uint32_t*>(j.mask);
      j.lvl = d->lvl;
      if (d->fb) j.fb = d->fb + (int64_t)b * d->fb_stride;
      if (d->nvis) j.nvis = d->nvis[b];
    }
  }
  *job = j;
}

// Lane step 4: another round while frontiers are left in the queue.
__global__ void k_batch_continue(cudaGraphConditionalHandle cond, const BatchDesc* d) {
  if (threadIdx.x == 0) {
    const int32_t head = *(volatile const int32_t*)&d->head;
    cudaGraphSetConditional(cond, head < d->B ? 1u : 0u);
  }
}

}  // namespace

// One lane's loop body.  sel_w != NULL (BFS only): the learned schedule; the
// work scan's last CTA picks push or pull per source and level, the push
// kernels and the pull kernel all follow and the ones not chosen return.
static int lane_launches(spmspv_handle* sub, BatchState* bs, int lane, int sem, bool bfs,
                         const Sched& sc, const float* sel_w, cudaGraphConditionalHandle cond,
                         cudaStream_t s) {
  k_batch_pop<<<1, 32, 0, s>>>(bs->desc, bs->jobs + lane);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "batch pop");
  const int k1_grid = sub->sm_count;
  if (bfs && sel_w) {
    SelArgs sa{};
    sa.w = sel_w;
    sa.allow_pull = 1;
    sa.bfs = 1;
    sa.lwb_lo = sub->lwb_lo;
    sa.direct_max = BFS_DIRECT_MAX;
    if ((e = launch_k1_bfs(sub->A, sub->ws, sub->nb_fine, nullptr, nullptr, k1_grid, nullptr, s,
                           nullptr, &sa)) != cudaSuccess)
      return cuda_fail(e, "batch work scan");
    if ((e = launch_k2(kMinSelect2nd, sub->A, sub->ws, sub->lwb_lo, sub->nb_fine, nullptr, 1,
                       sub->k2_grid, sub->k2_smem, s, 1, 0, BFS_DIRECT_MAX)) != cudaSuccess)
      return cuda_fail(e, "batch expand/scatter");
    const int lwb = sub->lwb_lo + 2;  // shared memory for the widest bucket
    const int nb_max = (int)(((int64_t)sub->A.m + (1 << sub->lwb_lo) - 1) >> sub->lwb_lo);
    const int k3_grid = std::max(1, std::min(nb_max, sub->sm_count * sub->k3_bps[2]));
    if ((e = launch_k3(kMinSelect2nd, true, sub->A, sub->ws, sub->lwb_lo, sub->nb_fine, nullptr,
                       nullptr, 0, nullptr, nullptr, k3_grid, k3_smem_bytes(lwb), s, 1,
                       BFS_DIRECT_MAX)) != cudaSuccess)
      return cuda_fail(e, "batch merge");
    if ((e = launch_pull_rows_lane(sub, sub->rows_sorted, s)) != cudaSuccess)
      return cuda_fail(e, "batch pull");
    k_batch_continue<<<1, 32, 0, s>>>(cond, bs->desc);
    return (e = cudaGetLastError()) == cudaSuccess ? SPMSPV_OK : cuda_fail(e, "batch condition");
  }
  if (bfs)
    e = launch_k1_bfs(sub->A, sub->ws, sub->nb_fine, nullptr, nullptr, k1_grid, &sc, s, nullptr);
  else
    e = launch_k1(sem, sub->A, sub->ws, sub->nb_fine, nullptr, nullptr, 0, nullptr, k1_grid, &sc, s,
                  nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "batch work scan");
  e = launch_k2(bfs ? kMinSelect2nd : sem, sub->A, sub->ws, sub->lwb_lo, sub->nb_fine, nullptr,
                1, sub->k2_grid, sub->k2_smem, s, 0, sc.q, bfs ? BFS_DIRECT_MAX : 0);
  if (e != cudaSuccess) return cuda_fail(e, "batch expand/scatter");
  const size_t k3_smem = k3_smem_bytes(sc.lwb);
  const int nb = (int)(((int64_t)sub->A.m + (1 << sc.lwb) - 1) >> sc.lwb);
  const int k3_grid = std::max(1, std::min(nb, sub->sm_count * sub->k3_bps[sc.lwb - sub->lwb_lo]));
  e = launch_k3(bfs ? kMinSelect2nd : sem, bfs, sub->A, sub->ws, sub->lwb_lo, sub->nb_fine, nullptr,
                nullptr, 0, nullptr, nullptr, k3_grid, k3_smem, s, 0, bfs ? BFS_DIRECT_MAX : 0);
  if (e != cudaSuccess) return cuda_fail(e, "batch merge");
  k_batch_continue<<<1, 32, 0, s>>>(cond, bs->desc);
  return (e = cudaGetLastError()) == cudaSuccess ? SPMSPV_OK : cuda_fail(e, "batch condition");
}

static int build_batch_graph(BatchState* bs, int sem, bool bfs, const Sched& sc,
                             const float* sel_w, int lanes, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
  int rc = SPMSPV_OK;
  if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) rc = cuda_fail(e, "stream");
  for (int l = 0; l < lanes && rc == SPMSPV_OK; ++l) {
    cudaGraphConditionalHandle cond;
    if ((e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess) {
      rc = cuda_fail(e, "lane handle");
      break;
    }
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np)) != cudaSuccess) {
      rc = cuda_fail(e, "lane node");
      break;
    }
    if ((e = cudaStreamBeginCaptureToGraph(cs, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
      rc = cuda_fail(e, "lane capture");
      break;
    }
    rc = lane_launches(bs->sub[l], bs, l, sem, bfs, sc, sel_w, cond, cs);
    cudaGraph_t tmp = nullptr;
    e = cudaStreamEndCapture(cs, &tmp);
    if (rc == SPMSPV_OK && e != cudaSuccess) rc = cuda_fail(e, "lane capture end");
  }
  if (rc == SPMSPV_OK && (e = cudaGraphInstantiate(&exec, g, 0)) != cudaSuccess)
    rc = cuda_fail(e, "instantiate batch graph");
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

static int ensure_batch(spmspv_handle* h, int lanes, BatchState** out) {
  BatchState* bs = (BatchState*)h->batch;
  if (!bs) {
    bs = new BatchState();
    memset(bs, 0, sizeof(*bs));
    cudaError_t e = cudaMalloc(&bs->jobs, sizeof(Job) * MAX_LANES);
    if (e == cudaSuccess) e = cudaMalloc(&bs->desc, sizeof(BatchDesc));
    if (e == cudaSuccess) e = cudaMemset(bs->desc, 0, sizeof(BatchDesc));
    if (e != cudaSuccess) {
      cudaFree(bs->jobs);
      cudaFree(bs->desc);
      delete bs;
      return fail(SPMSPV_ERR_OOM, "batch descriptors: %s", cudaGetErrorString(e));
    }
    h->batch = bs;
  }
  // one full workspace per lane, created like the parent handle
  for (int l = bs->lanes; l < lanes; ++l) {
    spmspv_handle* sub = nullptr;
    const int vt = h->A.val ? SPMSPV_VAL_F32 : SPMSPV_VAL_NONE;
    const uint32_t fl = h->flags & ~SPMSPV_CSC_PATTERN_SYMMETRIC;
    int rc = h->A.jc ? spmspv_create_dcsc(&sub, h->A.m, h->A.n, h->A.nnz, h->A.nzc, h->A.jc, h->A.colptr,
                                          h->A.rowidx, h->A.val, vt, fl)
                     : spmspv_create_csc(&sub, h->A.m, h->A.n, h->A.nnz, h->A.colptr, h->A.rowidx, h->A.val,
                                         vt, fl);
    if (rc != SPMSPV_OK) return rc;
    sub->ws.job = bs->jobs + l;
    cudaFree(sub->ws.ydense);  // the lanes never run the direct (+,*) form
    sub->ws.ydense = nullptr;
    bs->sub[l] = sub;
    bs->lanes = l + 1;
  }
  *out = bs;
  return SPMSPV_OK;
}

void release_batch(spmspv_handle* h) {
  BatchState* bs = (BatchState*)h->batch;
  if (!bs) return;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b <= SPMSPV_NUM_SCHEDULES; ++b)
      for (int c = 0; c < 2; ++c)
        for (int d = 0; d <= MAX_LANES; ++d)
          if (bs->graphs[a][b][c][d]) cudaGraphExecDestroy(bs->graphs[a][b][c][d]);
  for (int l = 0; l < bs->lanes; ++l) spmspv_destroy(bs->sub[l]);
  cudaFree(bs->jobs);
  cudaFree(bs->desc);
  delete bs;
  h->batch = nullptr;
}

int run_batched(spmspv_handle* h, int sem, bool bfs, int32_t B, const BatchDesc& v, uint32_t opts,
                int32_t lanes, cudaStream_t s);
int batch_set_level(spmspv_handle* h, int32_t lvl, cudaStream_t s);
int ensure_batch_state(spmspv_handle* h, int lanes);

int run_batched(spmspv_handle* h, int sem, bool bfs, int32_t B, const BatchDesc& v, uint32_t opts,
                int32_t lanes, cudaStream_t s) {
  if (lanes < 1 || lanes > MAX_LANES) return fail(SPMSPV_ERR_ARG, "lanes must be in [1, %d]", MAX_LANES);
  int sid = h->default_sched;
  if (opts & SPMSPV_SCHED_FORCE) sid = (int)SPMSPV_SCHED_ID(opts);
  if (sid >= 6) sid -= 6;  // the lanes run the push form (the learned BFS may pull)
  // learned BFS: the selector picks push or pull per source and level
  const bool learned = bfs && (opts & SPMSPV_SCHED_AUTO) && h->sel_w && h->sel_ready &&
                       pull_available(h, kMinSelect2nd);
  BatchState* bs = nullptr;
  int rc = ensure_batch(h, lanes, &bs);
  if (rc) return rc;
  if (learned) {
    for (int l = 0; l < lanes; ++l) {
      if (bs->sub[l]->xbits) continue;
      cudaError_t e = alloc_pull_buffers(bs->sub[l]);
      if (e != cudaSuccess) return cuda_fail(e, "lane pull buffers");
    }
  }
  const Sched sc = decode_schedule(h, sid);
  const int slot = learned ? SPMSPV_NUM_SCHEDULES : sid;
  cudaGraphExec_t& g = bs->graphs[bfs ? 1 : sem][slot][bfs ? 1 : 0][lanes];
  if (!g) {
    if ((rc = build_batch_graph(bs, bfs ? kMinSelect2nd : sem, bfs, sc, learned ? h->sel_w : nullptr,
                                lanes, &g)) != SPMSPV_OK)
      return rc;
  }
  k_batch_start<<<1, 32, 0, s>>>(bs->desc, v);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "batch start");
  if ((e = cudaGraphLaunch(g, s)) != cudaSuccess) return cuda_fail(e, "batch graph launch");
  h->last_stream = s;
  return SPMSPV_OK;
}

uint32_t batch_collect_status(spmspv_handle* h, cudaError_t* e) {
  *e = cudaSuccess;
  BatchState* bs = (BatchState*)h->batch;
  if (!bs) return 0u;
  uint32_t all = 0u;
  for (int l = 0; l < bs->lanes; ++l) {
    uint32_t v = 0u, z = 0u;
    if ((*e = cudaMemcpy(&v, &bs->sub[l]->ws.st->status, sizeof(v), cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (*e = cudaMemcpy(&bs->sub[l]->ws.st->status, &z, sizeof(z), cudaMemcpyHostToDevice)) != cudaSuccess)
      return all;
    all |= v;
  }
  return all;
}

int batch_set_level(spmspv_handle* h, int32_t lvl, cudaStream_t s) {
  BatchState* bs = (BatchState*)h->batch;
  k_batch_set_level<<<1, 32, 0, s>>>(bs->desc, lvl);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPMSPV_OK : cuda_fail(e, "batch level");
}

int ensure_batch_state(spmspv_handle* h, int lanes) {
  BatchState* bs = nullptr;
  return ensure_batch(h, lanes, &bs);
}

}  // namespace spmspv

using namespace spmspv;

extern "C" int spmspv_run_batched(spmspv_handle* h, int semiring, int32_t B, const int32_t* x_off,
                                  const int32_t* x_cnt, const int32_t* x_idx, const void* x_val,
                                  const uint32_t* masks, int64_t mask_stride, uint32_t opts,
                                  const int32_t* y_off, const int32_t* y_cap, int32_t* y_idx,
                                  void* y_val, int32_t* d_nnz_y, int32_t lanes,
                                  spmspv_stream_t stream) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (semiring < 0 || semiring > 2) return fail(SPMSPV_ERR_ARG, "unknown semiring %d", semiring);
  if (B < 0) return fail(SPMSPV_ERR_ARG, "B < 0");
  if (B == 0) return SPMSPV_OK;
  if (!x_off || !x_cnt || !x_idx || !y_off || !y_cap || !y_idx || !d_nnz_y)
    return fail(SPMSPV_ERR_ARG, "NULL batch array");
  if (semiring != SPMSPV_OR_AND_BOOL && (!x_val || !y_val)) return fail(SPMSPV_ERR_ARG, "x_val/y_val NULL");
  if (masks && mask_stride < ((int64_t)h->A.m + 31) / 32) return fail(SPMSPV_ERR_ARG, "mask_stride too small");
  BatchDesc v;
  memset(&v, 0, sizeof(v));
  v.B = B;
  v.x_off = x_off;
  v.x_cnt = x_cnt;
  v.x_idx = x_idx;
  v.x_val = (const uint32_t*)x_val;
  v.masks = masks;
  v.mask_stride = mask_stride;
  v.y_off = y_off;
  v.y_cap = y_cap;
  v.y_idx = y_idx;
  v.y_val = (uint32_t*)y_val;
  v.d_nnz_y = d_nnz_y;
  (void)(opts & SPMSPV_MASK_COMPLEMENT);
  if (masks && !(opts & SPMSPV_MASK_COMPLEMENT))
    return fail(SPMSPV_ERR_UNSUPPORTED, "batched masks are complemented masks");
  cudaStream_t s = (cudaStream_t)stream;
  auto persistent = [&](uint32_t o) {
    return run_batched_k6(h, semiring, B, x_off, x_cnt, x_idx, (const uint32_t*)x_val, masks, mask_stride, o,
                          y_off, y_cap, y_idx, (uint32_t*)y_val, d_nnz_y, s);
  };
  if (lanes == SPMSPV_LANES_PERSISTENT) return persistent(opts);
  if (lanes != 0) return run_batched(h, semiring, false, B, v, opts, lanes, s);
  // autotuned (persistent form): the profile needs the total frontier length
  std::vector<int32_t> cnt(B);
  cudaError_t e = cudaMemcpyAsync(cnt.data(), x_cnt, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "batch profile");
  int64_t total = 0;
  for (int32_t c : cnt) total += c;
  const uint32_t base = opts & ~(uint32_t)(SPMSPV_SCHED_FORCE | SPMSPV_SCHED_AUTO | SPMSPV_SCHED_OPT(0xFFu));
  return tune_and_run(
      h, tune_key(0, semiring, masks != nullptr, B, total), s,
      [&](int32_t ln, uint32_t so) {
        return ln == 0 ? persistent(base | so) : run_batched(h, semiring, false, B, v, base | so, ln, s);
      },
      SPMSPV_NUM_SCHEDULES / 2, kTunePersistent);
}

// ---------------------------------------------------------------------------
// Multi-source BFS: one batched (min, select2nd) step per level, every source
// with its own frontier, visited bitmap and outputs.
// ---------------------------------------------------------------------------
namespace spmspv {
namespace {

__global__ void k_msbfs_init(int32_t B, int32_t n, const int32_t* __restrict__ sources,
                             int32_t* __restrict__ level, int32_t* __restrict__ parent,
                             uint32_t* __restrict__ visited, int64_t vwords,
                             int32_t* __restrict__ fronts, int32_t* __restrict__ x_off,
                             int32_t* __restrict__ x_cnt, int32_t* __restrict__ y_off,
                             int32_t* __restrict__ y_cap, uint32_t* __restrict__ fb) {
  const int64_t total = (int64_t)B * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    level[i] = -1;
    parent[i] = -1;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)B * vwords;
       i += (int64_t)gridDim.x * blockDim.x)
    visited[i] = 0u;
  if (fb)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * (int64_t)B * vwords;
         i += (int64_t)gridDim.x * blockDim.x)
      fb[i] = 0u;
}

__global__ void k_msbfs_seed(int32_t B, int32_t n, const int32_t* __restrict__ sources,
                             int32_t* __restrict__ level, int32_t* __restrict__ parent,
                             uint32_t* __restrict__ visited, int64_t vwords,
                             int32_t* __restrict__ fronts, int32_t* __restrict__ x_off,
                             int32_t* __restrict__ x_cnt, int32_t* __restrict__ y_off,
                             int32_t* __restrict__ y_cap, int32_t* __restrict__ status,
                             uint32_t* __restrict__ fb, int32_t* __restrict__ nvis) {
  for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    const int32_t s = sources[b];
    x_off[b] = (int32_t)0;
    y_off[b] = 0;
    y_cap[b] = n;
    x_cnt[b] = 0;
    if (nvis) nvis[b] = 0;
    if (s < 0 || s >= n) {
      atomicOr(status, 1);
      continue;
    }
    level[(int64_t)b * n + s] = 0;
    parent[(int64_t)b * n + s] = s;
    visited[(int64_t)b * vwords + (s >> 5)] |= 1u << (s & 31);
    fronts[(int64_t)b * n] = s;
    x_cnt[b] = 1;
    if (fb) fb[2 * (int64_t)b * vwords + (s >> 5)] = 1u << (s & 31);  // level 0's frontier
    if (nvis) nvis[b] = 1;
  }
}

__global__ void k_msbfs_next(int32_t B, const int32_t* __restrict__ nnz, int32_t* __restrict__ x_cnt,
                             int32_t* __restrict__ total, int32_t* __restrict__ nvis) {
  int32_t t = 0;
  for (int32_t b = threadIdx.x; b < B; b += blockDim.x) {
    x_cnt[b] = nnz[b];
    if (nvis) nvis[b] += nnz[b];
    t += nnz[b];
  }
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(total, t);
}

// The persistent form's level update: y_b of the batched product holds the
// vertices source b reaches first at level L (the unvisited rows), each with
// its smallest frontier neighbour as value; they get their level, parent and
// visited bit, and y_b is the next frontier.
__global__ void k_msbfs_apply(int32_t B, int32_t n, int32_t L, const int32_t* __restrict__ y_idx,
                              const int32_t* __restrict__ y_par, const int32_t* __restrict__ nnz,
                              int32_t* __restrict__ level, int32_t* __restrict__ parent,
                              uint32_t* __restrict__ visited, int64_t vwords) {
  const int32_t b = blockIdx.y;
  if (b >= B) return;
  const int32_t c = nnz[b];
  const int64_t base = (int64_t)b * n;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < c; k += gridDim.x * blockDim.x) {
    const int32_t v = y_idx[base + k];
    level[base + v] = L;
    parent[base + v] = y_par[base + k];
    atomicOr(visited + (int64_t)b * vwords + (v >> 5), 1u << (v & 31));
  }
}

// The learned schedule of the persistent form.  k_msbfs_stats gathers each
// source's level features as a single call would compute them (products,
// entries with a non-empty column, the largest column; several CTAs per
// source), k_msbfs_decide (one warp per source) adds the frontier size and
// the vertices reached, evaluates the network and clears the statistics for
// the next level; a level of at most BFS_DIRECT_MAX products stays push.  A
// pull choice keeps the source out of the batched product (its push count
// is 0); k_msbfs_setbits sets its frontier in its bitmap for k_msbfs_pull.
__global__ void __launch_bounds__(256)
k_msbfs_stats(int32_t B, int32_t n, const int32_t* __restrict__ colptr, const int32_t* __restrict__ fronts,
              const int32_t* __restrict__ x_cnt, unsigned long long* __restrict__ wsum, int32_t* __restrict__ fcnt,
              int32_t* __restrict__ mdeg) {
  const int32_t b = blockIdx.y;
  if (b >= B) return;
  const int32_t f = x_cnt[b];
  const int32_t* x = fronts + (int64_t)b * n;
  unsigned long long W = 0;
  int32_t fc = 0, md = 0;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < f; k += gridDim.x * blockDim.x) {
    const int32_t j = x[k];
    const int32_t d = colptr[j + 1] - colptr[j];
    W += (unsigned long long)d;
    fc += d > 0;
    md = max(md, d);
  }
  for (int o = 16; o > 0; o >>= 1) {
    W += __shfl_xor_sync(0xffffffffu, W, o);
    fc += __shfl_xor_sync(0xffffffffu, fc, o);
    md = max(md, __shfl_xor_sync(0xffffffffu, md, o));
  }
  if ((threadIdx.x & 31) == 0 && W > 0) {
    atomicAdd(wsum + b, W);
    atomicAdd(fcnt + b, fc);
    atomicMax(mdeg + b, md);
  }
}

__global__ void k_msbfs_decide(int32_t B, int32_t n, int64_t nnz, const float* __restrict__ w,
                               const int32_t* __restrict__ x_cnt, const int32_t* __restrict__ nvis,
                               unsigned long long* __restrict__ wsum, int32_t* __restrict__ fcnt,
                               int32_t* __restrict__ mdeg, int32_t* __restrict__ xc_push, int32_t* __restrict__ dir,
                               int32_t* __restrict__ pcnt) {
  const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= B) return;  // the whole warp
  const int lane = threadIdx.x & 31;
  const int32_t f = x_cnt[b];
  const long long W = (long long)wsum[b];
  int d = 0;
  if (f > 0 && W > BFS_DIRECT_MAX) {
    float xf[SEL_IN];
    sel_features_of(f, (int32_t)min(W, (long long)INT32_MAX), fcnt[b], mdeg[b], nvis[b], n, n, nnz, xf);
    d = sel_pick_warp(w, xf, 1) >= SPMSPV_NUM_SCHEDULES / 2 ? 1 : 0;
  }
  if (lane == 0) {
    dir[b] = d;
    xc_push[b] = d ? 0 : f;
    pcnt[b] = 0;
    wsum[b] = 0ull;
    fcnt[b] = 0;
    mdeg[b] = 0;
  }
}

__global__ void __launch_bounds__(256)
k_msbfs_setbits(int32_t B, int32_t n, const int32_t* __restrict__ dir, const int32_t* __restrict__ fronts,
                const int32_t* __restrict__ x_cnt, uint32_t* __restrict__ fbits, int64_t vwords) {
  const int32_t b = blockIdx.y;
  if (b >= B || !dir[b]) return;
  const int32_t f = x_cnt[b];
  const int32_t* x = fronts + (int64_t)b * n;
  uint32_t* fb = fbits + (int64_t)b * vwords;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < f; k += gridDim.x * blockDim.x)
    atomicOr(fb + (x[k] >> 5), 1u << (x[k] & 31));
}

// A pull level of the persistent form for every source that chose pull
// (Sec. II-B's matrix-driven form): a thread owns one 32-vertex word of the
// source's visited bitmap, every unvisited vertex scans its neighbours (its
// column: the pattern is symmetric) for members of the source's frontier
// and takes the smallest (the first when row ids ascend in every column);
// the vertices found get level, parent and visited bit and are appended to
// the next frontier, whose order the next level does not depend on.
__global__ void __launch_bounds__(256)
k_msbfs_pull(int32_t B, int32_t n, int32_t L, const int32_t* __restrict__ colptr, const int32_t* __restrict__ rowidx,
             int rows_sorted, const int32_t* __restrict__ dir, const uint32_t* __restrict__ fbits, int64_t vwords,
             uint32_t* __restrict__ visited, int32_t* __restrict__ level, int32_t* __restrict__ parent,
             int32_t* __restrict__ nxt, int32_t* __restrict__ pcnt) {
  const int32_t b = blockIdx.y;
  if (b >= B || !dir[b]) return;
  const int lane = threadIdx.x & 31;
  const int64_t base = (int64_t)b * n;
  const uint32_t* fb = fbits + (int64_t)b * vwords;
  uint32_t* vis = visited + (int64_t)b * vwords;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); w0 < vwords; w0 += stride) {
    const int64_t w = w0 + lane;
    uint32_t allowed = 0u;
    if (w < vwords) {
      allowed = ~vis[w];
      const int32_t r0 = (int32_t)(w * 32);
      if (n - r0 < 32) allowed &= (1u << (n - r0)) - 1u;
    }
    uint32_t found = 0u;
    while (allowed) {
      const int k = __ffs(allowed) - 1;
      allowed &= allowed - 1u;
      const int32_t r = (int32_t)(w * 32) + k;
      int32_t best = INT32_MAX;
      for (int32_t p = colptr[r], p1 = colptr[r + 1]; p < p1; ++p) {
        const int32_t j = rowidx[p];
        if (!((fb[j >> 5] >> (j & 31)) & 1u)) continue;
        best = min(best, j);
        if (rows_sorted) break;
      }
      if (best != INT32_MAX) {
        found |= 1u << k;
        level[base + r] = L;
        parent[base + r] = best;
      }
    }
    if (found) vis[w] |= found;
    // one reservation per warp, then the new vertices
    const int32_t c = __popc(found);
    int32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    int32_t pos = 0;
    if (lane == 31 && incl > 0) pos = atomicAdd(pcnt + b, incl);
    pos = __shfl_sync(0xffffffffu, pos, 31) + incl - c;
    for (uint32_t bits = found; bits; bits &= bits - 1u) nxt[base + pos++] = (int32_t)(w * 32) + __ffs(bits) - 1;
  }
}

// After a pull level: the source's frontier bitmap cleared (all of it,
// several CTAs per source) and its count of new vertices moved to nnz.
__global__ void __launch_bounds__(256)
k_msbfs_pull_done(int32_t B, const int32_t* __restrict__ dir, const int32_t* __restrict__ pcnt,
                  uint32_t* __restrict__ fbits, int64_t vwords, int32_t* __restrict__ nnz) {
  const int32_t b = blockIdx.y;
  if (b >= B || !dir[b]) return;
  uint32_t* fb = fbits + (int64_t)b * vwords;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < vwords; i += (int64_t)gridDim.x * blockDim.x)
    fb[i] = 0u;
  if (blockIdx.x == 0 && threadIdx.x == 0) nnz[b] = pcnt[b];
}

}  // namespace
}  // namespace spmspv

static int msbfs_run(spmspv_handle* h, int32_t B, const int32_t* sources, int32_t* level,
                     int32_t* parent, int32_t* nlevels, uint32_t opts, int32_t lanes,
                     spmspv_stream_t stream) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (h->A.m != h->A.n) return fail(SPMSPV_ERR_ARG, "BFS needs a square matrix");
  if (B < 1 || !sources || !level || !parent) return fail(SPMSPV_ERR_ARG, "bad multi-source BFS arguments");
  if (B > (int32_t)(((int64_t)1 << 31) / h->A.n))
    return fail(SPMSPV_ERR_UNSUPPORTED, "B * n must stay below 2^31");
  cudaStream_t s = (cudaStream_t)stream;
  const int32_t n = h->A.n;
  const int64_t vwords = ((int64_t)n + 31) / 32;
  // the learned schedule (push or pull per source and level) needs the
  // selector's weights and a pattern-symmetric matrix
  // the learned schedule: push or pull per source and level (in the lanes,
  // or around the persistent form's push launch)
  const bool persistent = lanes == SPMSPV_LANES_PERSISTENT;
  const bool learned = (opts & SPMSPV_SCHED_AUTO) && h->sel_w && h->sel_ready &&
                       pull_available(h, kMinSelect2nd);
  // per-source frontiers, visited bitmaps and batch arrays (freed on return);
  // the persistent form writes each level's product to a second frontier
  // array with the parents beside it
  int32_t *fronts = nullptr, *arr = nullptr, *fronts2 = nullptr, *ypar = nullptr;
  uint32_t *visited = nullptr, *fbs = nullptr;
  unsigned long long* wsum = nullptr;
  cudaError_t e = cudaMalloc(&fronts, sizeof(int32_t) * (size_t)B * n);
  if (e == cudaSuccess) e = cudaMalloc(&visited, sizeof(uint32_t) * (size_t)B * vwords);
  if (e == cudaSuccess) e = cudaMalloc(&arr, sizeof(int32_t) * ((size_t)B * 11 + 8));
  if (e == cudaSuccess && persistent && learned) e = cudaMalloc(&wsum, sizeof(unsigned long long) * (size_t)B);
  // frontier bitmaps of the learned schedule: two per source in the lanes
  // (this level's and the next), one in the persistent form
  const size_t fb_words = (persistent ? 1 : 2) * (size_t)B * vwords;
  if (e == cudaSuccess && learned) e = cudaMalloc(&fbs, sizeof(uint32_t) * fb_words);
  if (e == cudaSuccess && persistent) e = cudaMalloc(&fronts2, sizeof(int32_t) * (size_t)B * n);
  if (e == cudaSuccess && persistent) e = cudaMalloc(&ypar, sizeof(int32_t) * (size_t)B * n);
  auto release = [&]() {
    cudaFree(fronts);
    cudaFree(visited);
    cudaFree(arr);
    cudaFree(fbs);
    cudaFree(fronts2);
    cudaFree(ypar);
    cudaFree(wsum);
  };
  if (e != cudaSuccess) {
    release();
    cudaGetLastError();
    return fail(SPMSPV_ERR_OOM, "multi-source BFS buffers: %s", cudaGetErrorString(e));
  }
  int32_t* x_off = arr;
  int32_t* x_cnt = arr + B;
  int32_t* y_off = arr + 2 * B;
  int32_t* y_cap = arr + 3 * B;
  int32_t* nnz = arr + 4 * B;
  int32_t* nvis = learned ? arr + 5 * B : nullptr;
  int32_t* xc_push = arr + 6 * B;  // persistent + learned: push counts, direction, pull counts
  int32_t* dir = arr + 7 * B;
  int32_t* pcnt = arr + 8 * B;
  int32_t* fcnt = arr + 9 * B;  // persistent + learned: level statistics
  int32_t* mdeg = arr + 10 * B;
  int32_t* misc = arr + 11 * B;  // [0] status, [1] frontier total
  // frontier b lives at fronts + b*n: express the offsets relative to fronts
  cudaMemsetAsync(misc, 0, sizeof(int32_t) * 8, s);
  const int grid = h->sm_count * 4;
  uint32_t* fb_lanes = persistent ? nullptr : fbs;
  if (persistent && fbs) cudaMemsetAsync(fbs, 0, sizeof(uint32_t) * fb_words, s);
  if (wsum) {
    cudaMemsetAsync(wsum, 0, sizeof(unsigned long long) * B, s);
    cudaMemsetAsync(fcnt, 0, sizeof(int32_t) * 2 * B, s);
  }
  k_msbfs_init<<<grid, 256, 0, s>>>(B, n, sources, level, parent, visited, vwords, fronts, x_off,
                                    x_cnt, y_off, y_cap, fb_lanes);
  k_msbfs_seed<<<(B + 255) / 256, 256, 0, s>>>(B, n, sources, level, parent, visited, vwords, fronts,
                                               x_off, x_cnt, y_off, y_cap, misc, fb_lanes, nvis);
  // offsets: frontier b starts at b*n
  {
    std::vector<int32_t> off(B);
    for (int32_t b = 0; b < B; ++b) off[b] = b * n;
    cudaMemcpyAsync(x_off, off.data(), sizeof(int32_t) * B, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(y_off, off.data(), sizeof(int32_t) * B, cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
  }
  BatchDesc v;
  memset(&v, 0, sizeof(v));
  v.B = B;
  v.x_off = x_off;
  v.x_cnt = x_cnt;
  v.x_idx = fronts;
  v.masks = visited;
  v.mask_stride = vwords;
  v.y_off = y_off;
  v.y_cap = y_cap;
  v.y_idx = fronts;
  v.d_nnz_y = nnz;
  v.level = level;
  v.parent = parent;
  v.vstride = n;
  v.fb = fbs;
  v.fb_stride = 2 * vwords;
  v.nvis = nvis;
  int32_t L = 0;
  rc = SPMSPV_OK;
  if (persistent) {
    // level L: y_b = A x_b under the complement of visited_b, x_b = the
    // frontier with its vertex ids as values, so y_b(i) is the smallest
    // frontier neighbour of every vertex first reached at L; with the
    // learned schedule the sources that chose pull leave the batched product
    // to k_msbfs_pull
    int32_t* cur = fronts;
    int32_t* nxt = fronts2;
    // pull: one 32-vertex word per thread, up to 64 CTAs per source (more
    // when there are few sources)
    const int64_t pull_cap = std::max<int64_t>(64, ((int64_t)h->sm_count * 8 + B - 1) / B);
    const int pull_grid = (int)std::min<int64_t>((vwords + 255) / 256, pull_cap);
    // the per-source helpers: enough CTAs per source for about 8 per SM
    const int per_src = (int)std::max<int64_t>(1, std::min<int64_t>(256, ((int64_t)h->sm_count * 8 + B - 1) / B));
    for (L = 1; L <= n; ++L) {
      for (int32_t b0 = 0; learned && b0 < B; b0 += 65535) {
        const int32_t bc = std::min<int32_t>(B - b0, 65535);
        k_msbfs_stats<<<dim3(per_src, bc), 256, 0, s>>>(bc, n, h->A.colptr, cur + (int64_t)b0 * n, x_cnt + b0,
                                                         wsum + b0, fcnt + b0, mdeg + b0);
        k_msbfs_decide<<<(bc + 7) / 8, 256, 0, s>>>(bc, n, h->A.nnz, h->sel_w, x_cnt + b0, nvis + b0, wsum + b0,
                                                    fcnt + b0, mdeg + b0, xc_push + b0, dir + b0, pcnt + b0);
        k_msbfs_setbits<<<dim3(per_src, bc), 256, 0, s>>>(bc, n, dir + b0, cur + (int64_t)b0 * n, x_cnt + b0,
                                                           fbs + (int64_t)b0 * vwords, vwords);
      }
      if ((rc = run_batched_k6(h, kMinSelect2nd, B, x_off, learned ? xc_push : x_cnt, cur, (const uint32_t*)cur,
                               visited, vwords, opts, y_off, y_cap, nxt, (uint32_t*)ypar, nnz, s, true)) !=
          SPMSPV_OK)
        break;
      for (int32_t b0 = 0; b0 < B; b0 += 65535)
        k_msbfs_apply<<<dim3(16, (unsigned)std::min<int32_t>(B - b0, 65535)), 256, 0, s>>>(
            B - b0, n, L, nxt + (int64_t)b0 * n, ypar + (int64_t)b0 * n, nnz + b0, level + (int64_t)b0 * n,
            parent + (int64_t)b0 * n, visited + (int64_t)b0 * vwords, vwords);
      for (int32_t b0 = 0; learned && b0 < B; b0 += 65535) {
        const unsigned gy = (unsigned)std::min<int32_t>(B - b0, 65535);
        k_msbfs_pull<<<dim3(pull_grid, gy), 256, 0, s>>>(
            B - b0, n, L, h->A.colptr, h->A.rowidx, h->rows_sorted, dir + b0, fbs + (int64_t)b0 * vwords, vwords,
            visited + (int64_t)b0 * vwords, level + (int64_t)b0 * n, parent + (int64_t)b0 * n,
            nxt + (int64_t)b0 * n, pcnt + b0);
        k_msbfs_pull_done<<<dim3(per_src, gy), 256, 0, s>>>(B - b0, dir + b0, pcnt + b0, fbs + (int64_t)b0 * vwords,
                                                             vwords, nnz + b0);
      }
      cudaMemsetAsync(misc + 1, 0, sizeof(int32_t), s);
      k_msbfs_next<<<1, 1024, 0, s>>>(B, nnz, x_cnt, misc + 1, nvis);
      int32_t total = 0;
      e = cudaMemcpyAsync(&total, misc + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        rc = cuda_fail(e, "multi-source BFS level");
        break;
      }
      std::swap(cur, nxt);
      if (total == 0) break;
    }
  } else if ((rc = ensure_batch_state(h, lanes)) == SPMSPV_OK) {
    for (L = 1; L <= n; ++L) {
      if ((rc = batch_set_level(h, L, s)) != SPMSPV_OK) break;
      if ((rc = run_batched(h, kMinSelect2nd, true, B, v, opts, lanes, s)) != SPMSPV_OK) break;
      cudaMemsetAsync(misc + 1, 0, sizeof(int32_t), s);
      k_msbfs_next<<<1, 1024, 0, s>>>(B, nnz, x_cnt, misc + 1, nvis);
      int32_t total = 0;
      e = cudaMemcpyAsync(&total, misc + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        rc = cuda_fail(e, "multi-source BFS level");
        break;
      }
      if (total == 0) break;
    }
  }
  if (rc == SPMSPV_OK && nlevels) {
    e = cudaMemcpyAsync(nlevels, &L, sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "level count");
  }
  cudaStreamSynchronize(s);
  release();
  return rc;
}

// ---------------------------------------------------------------------------
// Andersen-Chung-Lang local clustering (Sec. I names it a one-SpMSpV-per-step
// customer; the paper gives no algorithm).  Synchronous push per seed b with
// residual r_b and approximate PageRank p_b (dense, n each), unweighted A,
// degree d(u) = column length:
//   S = {u : r(u) >= eps * d(u)}; for u in S: x(u) = (1-alpha) r(u) / (2 d(u)),
//   p(u) += alpha r(u), r(u) = (1-alpha) r(u) / 2; then r += A x.
// The next S is drawn only from the rows the step touched (y) and the last S.
// ---------------------------------------------------------------------------
namespace spmspv {
namespace {

__global__ void k_acl_init(int64_t total, float* __restrict__ R, float* __restrict__ P) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    R[i] = 0.f;
    P[i] = 0.f;
  }
}

__global__ void k_acl_seed(int32_t B, int32_t n, const int32_t* __restrict__ seeds,
                           const int32_t* __restrict__ colptr, float eps, float* __restrict__ R,
                           int32_t* __restrict__ act, int32_t* __restrict__ cnt,
                           int32_t* __restrict__ status) {
  for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    const int32_t s = seeds[b];
    cnt[b] = 0;
    if (s < 0 || s >= n) {
      atomicOr(status, 1);
      continue;
    }
    R[(int64_t)b * n + s] = 1.f;
    const int32_t d = colptr[s + 1] - colptr[s];
    if (d > 0 && 1.f >= eps * (float)d) {
      act[(int64_t)b * n] = s;
      cnt[b] = 1;
    }
  }
}

// Push the active set: x values, p += alpha r, r = (1-alpha) r / 2.
__global__ void k_acl_push(int32_t B, int32_t n, const int32_t* __restrict__ colptr, float alpha,
                           const int32_t* __restrict__ act, const int32_t* __restrict__ cnt,
                           float* __restrict__ xv, float* __restrict__ R, float* __restrict__ P) {
  const int32_t b = blockIdx.y;
  const int32_t c = cnt[b];
  const int64_t base = (int64_t)b * n;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < c; k += gridDim.x * blockDim.x) {
    const int32_t u = act[base + k];
    const float r = R[base + u];
    const float d = (float)(colptr[u + 1] - colptr[u]);
    xv[base + k] = (1.f - alpha) * r / (2.f * d);
    P[base + u] += alpha * r;
    R[base + u] = (1.f - alpha) * r * 0.5f;
  }
}

// r += y for every seed's product.
__global__ void k_acl_add(int32_t B, int32_t n, const int32_t* __restrict__ y_idx,
                          const float* __restrict__ y_val, const int32_t* __restrict__ ny,
                          float* __restrict__ R) {
  const int32_t b = blockIdx.y;
  const int32_t c = ny[b];
  const int64_t base = (int64_t)b * n;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < c; k += gridDim.x * blockDim.x)
    R[base + y_idx[base + k]] += y_val[base + k];
}

// Next active set from the candidates y_b and the last S_b (deduplicated with
// a per-seed bitmap that is cleared again by k_acl_unmark).
__global__ void k_acl_select(int32_t B, int32_t n, int64_t words, const int32_t* __restrict__ colptr,
                             float eps, const int32_t* __restrict__ y_idx, const int32_t* __restrict__ ny,
                             const int32_t* __restrict__ act, const int32_t* __restrict__ cnt,
                             const float* __restrict__ R, uint32_t* __restrict__ mark,
                             int32_t* __restrict__ nact, int32_t* __restrict__ ncnt) {
  const int32_t b = blockIdx.y;
  const int64_t base = (int64_t)b * n;
  const int32_t c1 = ny[b], c2 = cnt[b];
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < c1 + c2; k += gridDim.x * blockDim.x) {
    const int32_t u = k < c1 ? y_idx[base + k] : act[base + (k - c1)];
    const float d = (float)(colptr[u + 1] - colptr[u]);
    if (!(d > 0.f) || R[base + u] < eps * d) continue;
    const uint32_t bit = 1u << (u & 31);
    const uint32_t old = atomicOr(mark + (int64_t)b * words + (u >> 5), bit);
    if (old & bit) continue;
    const int32_t pos = atomicAdd(ncnt + b, 1);
    nact[base + pos] = u;
  }
}

__global__ void k_acl_unmark(int32_t B, int32_t n, int64_t words, const int32_t* __restrict__ nact,
                             const int32_t* __restrict__ ncnt, uint32_t* __restrict__ mark,
                             int32_t* __restrict__ total) {
  const int32_t b = blockIdx.y;
  const int32_t c = ncnt[b];
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < c; k += gridDim.x * blockDim.x) {
    const int32_t u = nact[(int64_t)b * n + k];
    mark[(int64_t)b * words + (u >> 5)] = 0u;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && c) atomicAdd(total, c);
}

}  // namespace
}  // namespace spmspv

static int acl_run(spmspv_handle* h, int32_t B, const int32_t* seeds, float alpha, float eps,
                   int32_t max_steps, float* p_out, float* r_out, int32_t* steps_out, uint32_t opts,
                   int32_t lanes, spmspv_stream_t stream) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (h->A.m != h->A.n) return fail(SPMSPV_ERR_ARG, "ACL needs a square matrix");
  if (h->A.jc) return fail(SPMSPV_ERR_UNSUPPORTED, "ACL reads vertex degrees from CSC column pointers");
  if (h->A.val) return fail(SPMSPV_ERR_ARG, "ACL uses the unweighted graph: create the handle with SPMSPV_VAL_NONE");
  if (B < 1 || !seeds || !p_out || !r_out) return fail(SPMSPV_ERR_ARG, "bad ACL arguments");
  if (!(alpha > 0.f && alpha < 1.f) || !(eps > 0.f) || max_steps < 0)
    return fail(SPMSPV_ERR_ARG, "need 0 < alpha < 1, eps > 0, max_steps >= 0");
  if (B > (int32_t)(((int64_t)1 << 31) / h->A.n)) return fail(SPMSPV_ERR_UNSUPPORTED, "B * n must stay below 2^31");
  if (B > 65535) return fail(SPMSPV_ERR_UNSUPPORTED, "at most 65535 seeds per call");
  cudaStream_t s = (cudaStream_t)stream;
  const int32_t n = h->A.n;
  const int64_t words = ((int64_t)n + 31) / 32;
  const size_t bn = (size_t)B * n;
  int32_t *act0 = nullptr, *act1 = nullptr, *yi = nullptr, *arr = nullptr;
  float *xv = nullptr, *yv = nullptr;
  uint32_t* mark = nullptr;
  cudaError_t e = cudaMalloc(&act0, sizeof(int32_t) * bn);
  if (e == cudaSuccess) e = cudaMalloc(&act1, sizeof(int32_t) * bn);
  if (e == cudaSuccess) e = cudaMalloc(&yi, sizeof(int32_t) * bn);
  if (e == cudaSuccess) e = cudaMalloc(&xv, sizeof(float) * bn);
  if (e == cudaSuccess) e = cudaMalloc(&yv, sizeof(float) * bn);
  if (e == cudaSuccess) e = cudaMalloc(&mark, sizeof(uint32_t) * (size_t)B * words);
  if (e == cudaSuccess) e = cudaMalloc(&arr, sizeof(int32_t) * ((size_t)B * 8 + 8));
  auto release = [&]() {
    cudaFree(act0); cudaFree(act1); cudaFree(yi); cudaFree(xv); cudaFree(yv); cudaFree(mark); cudaFree(arr);
  };
  if (e != cudaSuccess) {
    release();
    cudaGetLastError();
    return fail(SPMSPV_ERR_OOM, "ACL buffers: %s", cudaGetErrorString(e));
  }
  int32_t* cnt0 = arr;
  int32_t* cnt1 = arr + B;
  int32_t* ny = arr + 2 * B;
  int32_t* x_off = arr + 3 * B;
  int32_t* y_cap = arr + 4 * B;
  int32_t* misc = arr + 8 * B;  // [0] status [1] active total
  cudaMemsetAsync(mark, 0, sizeof(uint32_t) * (size_t)B * words, s);
  cudaMemsetAsync(misc, 0, sizeof(int32_t) * 8, s);
  {
    std::vector<int32_t> off(B), cap(B, n);
    for (int32_t b = 0; b < B; ++b) off[b] = b * n;
    cudaMemcpyAsync(x_off, off.data(), sizeof(int32_t) * B, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(y_cap, cap.data(), sizeof(int32_t) * B, cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
  }
  k_acl_init<<<h->sm_count * 4, 256, 0, s>>>((int64_t)bn, r_out, p_out);
  k_acl_seed<<<(B + 255) / 256, 256, 0, s>>>(B, n, seeds, h->A.colptr, eps, r_out, act0, cnt0, misc);
  // the persistent form: each step's products are one launch over every seed
  const bool persistent = lanes == SPMSPV_LANES_PERSISTENT;
  if (!persistent && (rc = ensure_batch_state(h, lanes)) != SPMSPV_OK) {
    release();
    return rc;
  }
  const dim3 g2(16, B);
  int32_t step = 0;
  int32_t* act = act0;
  int32_t* nact = act1;
  int32_t* cnt = cnt0;
  int32_t* ncnt = cnt1;
  for (step = 0; step < max_steps; ++step) {
    k_acl_push<<<g2, 256, 0, s>>>(B, n, h->A.colptr, alpha, act, cnt, xv, r_out, p_out);
    BatchDesc v;
    memset(&v, 0, sizeof(v));
    v.B = B;
    v.x_off = x_off;
    v.x_cnt = cnt;
    v.x_idx = act;
    v.x_val = (const uint32_t*)xv;
    v.y_off = x_off;
    v.y_cap = y_cap;
    v.y_idx = yi;
    v.y_val = (uint32_t*)yv;
    v.d_nnz_y = ny;
    rc = persistent ? run_batched_k6(h, kPlusTimes, B, x_off, cnt, act, (const uint32_t*)xv, nullptr, 0, opts,
                                     x_off, y_cap, yi, (uint32_t*)yv, ny, s)
                    : run_batched(h, kPlusTimes, false, B, v, opts, lanes, s);
    if (rc != SPMSPV_OK) break;
    k_acl_add<<<g2, 256, 0, s>>>(B, n, yi, yv, ny, r_out);
    cudaMemsetAsync(ncnt, 0, sizeof(int32_t) * B, s);
    cudaMemsetAsync(misc + 1, 0, sizeof(int32_t), s);
    k_acl_select<<<g2, 256, 0, s>>>(B, n, words, h->A.colptr, eps, yi, ny, act, cnt, r_out, mark, nact, ncnt);
    k_acl_unmark<<<g2, 256, 0, s>>>(B, n, words, nact, ncnt, mark, misc + 1);
    int32_t total = 0;
    e = cudaMemcpyAsync(&total, misc + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "ACL step");
      break;
    }
    std::swap(act, nact);
    std::swap(cnt, ncnt);
    if (total == 0) {
      ++step;
      break;
    }
  }
  if (rc == SPMSPV_OK && steps_out) {
    e = cudaMemcpyAsync(steps_out, &step, sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "ACL step count");
  }
  cudaStreamSynchronize(s);
  release();
  return rc;
}

// lanes == 0: the autotuner picks the form (lanes, or the persistent form,
// cached as lanes 0) and the schedule per (B) profile, timing whole runs (each
// run starts from its sources/seeds again, so reruns are harmless).
extern "C" int spmspv_msbfs(spmspv_handle* h, int32_t B, const int32_t* sources, int32_t* level,
                            int32_t* parent, int32_t* nlevels, uint32_t opts, int32_t lanes,
                            spmspv_stream_t stream) {
  if (lanes != 0) return msbfs_run(h, B, sources, level, parent, nlevels, opts, lanes, stream);
  int rc = check_handle(h);
  if (rc) return rc;
  if (opts & SPMSPV_SCHED_AUTO)  // the learned schedule: the form (lanes or persistent) is tuned
    return tune_and_run(h, tune_key(3, kMinSelect2nd, 1, B, 0), (cudaStream_t)stream,
                        [&](int32_t ln, uint32_t) {
                          return msbfs_run(h, B, sources, level, parent, nlevels, opts,
                                           ln == 0 ? SPMSPV_LANES_PERSISTENT : ln, stream);
                        },
                        1, kTuneBoth);
  const uint32_t base = opts & ~(uint32_t)(SPMSPV_SCHED_FORCE | SPMSPV_SCHED_AUTO | SPMSPV_SCHED_OPT(0xFFu));
  return tune_and_run(h, tune_key(1, kMinSelect2nd, 1, B, 0), (cudaStream_t)stream,
                      [&](int32_t ln, uint32_t so) {
                        return msbfs_run(h, B, sources, level, parent, nlevels, base | so,
                                         ln == 0 ? SPMSPV_LANES_PERSISTENT : ln, stream);
                      },
                      SPMSPV_NUM_SCHEDULES / 2, kTuneBoth);
}

extern "C" int spmspv_acl(spmspv_handle* h, int32_t B, const int32_t* seeds, float alpha, float eps,
                          int32_t max_steps, float* p_out, float* r_out, int32_t* steps_out,
                          int32_t lanes, spmspv_stream_t stream) {
  if (lanes != 0)
    return acl_run(h, B, seeds, alpha, eps, max_steps, p_out, r_out, steps_out, 0, lanes, stream);
  int rc = check_handle(h);
  if (rc) return rc;
  return tune_and_run(h, tune_key(2, kPlusTimes, 0, B, 0), (cudaStream_t)stream,
                      [&](int32_t ln, uint32_t so) {
                        return acl_run(h, B, seeds, alpha, eps, max_steps, p_out, r_out, steps_out, so,
                                       ln == 0 ? SPMSPV_LANES_PERSISTENT : ln, stream);
                      },
                      SPMSPV_NUM_SCHEDULES / 2, kTuneBoth);
}
