// The handle behind the opaque spmspv_handle of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>

#include "spmspv_internal.cuh"

constexpr uint32_t kHandleMagic = 0x53704d53u;
constexpr int MAX_LANES = 16;  // concurrent lanes of the batched form

struct spmspv_handle {
  uint32_t magic;
  int device;
  int sm_count;
  spmspv::Matrix A;
  uint32_t flags;
  int rows_sorted;      // row ids ascend inside every column
  int lwb_lo;           // log2 of the narrowest bucket width of the schedules
  int nb_fine;          // buckets at the narrowest width
  void* ws_base;
  size_t ws_bytes;
  spmspv::Workspace ws;
  size_t k2_smem;
  size_t k3_smem_max;
  int k2_grid;
  int k3_bps[3];        // K3 CTAs per SM for each of the three bucket widths
  int k1_grid_max;
  int k1_grid_dev;      // K1 CTAs when nnz(x) is only known on the device (BFS, lanes)
  int default_sched;
  cudaStream_t last_stream;
  int last_empty;
  int plus_direct;      // the current (+,*) call may run the direct form (ws.ydense, per call)
  const uint32_t* k1_mask;  // mask whose bits the work scan counts (features), or NULL
  void* prof;           // std::vector<ProfileCall>* while profiling, else NULL
  int32_t* rowidx_k2;   // owned row-id copy with hub rows relabelled (NULL without hubs)
  int32_t* dcsc_aux;    // owned auxiliary column index of a DCSC matrix (NULL for CSC)
  void* bfs_graph[SPMSPV_NUM_SCHEDULES + 2];  // cudaGraphExec_t per schedule (+ learned, + rule)
  // learned schedule selector
  int sel_ready;        // weights present
  float* sel_w;         // device weights (layout in selector.cu)
  void* batch;          // BatchState* of the batched lanes (batched.cu), lazily created
  void* k6;             // K6Buffers* of the persistent batched form (batched_k6.cu), lazily created
  void* tune;           // TuneCache* of the batched-form autotuner (autotune.cu), lazily created
  void* hostio;         // HostIO* of spmspv_run_host (host_io.cu), lazily created
  // pull direction (dense frontier) buffers, allocated on first use
  uint32_t* xbits;      // [ceil(n/32)] frontier bitmap
  uint32_t* xdense;     // [n] frontier values
  unsigned long long* pull_status;  // [row tiles] look-back words
  int pull_tiles;
  // BFS buffers, allocated on first use
  int32_t* bfs_front;   // [n] frontier list (x and y of each level)
  uint32_t* bfs_visited;  // [ceil(n/32)]
  uint32_t* bfs_fb;     // [2 * ceil(n/32)] frontier bitmaps (current / next level)
  int32_t* bfs_front2;  // [n] the persistent BFS kernel's second frontier buffer
  int32_t* bfs_slice;   // [3 * fused grid] its per-CTA slice sums
  int fused_grid;       // CTAs of the persistent BFS kernel (0: not available)
  // connected components (first use): frontier (x) and round output (y), counts
  int32_t* cc_x_idx;
  uint32_t* cc_x_val;
  int32_t* cc_y_idx;
  uint32_t* cc_y_val;
  int32_t* cc_cnt;
  void* cc_graph[SPMSPV_NUM_SCHEDULES / 2];  // cudaGraphExec_t per push schedule
  // maximal independent set (first use): candidates (x), SpMSpV output (y),
  // joiners, dense y lookup, decided bitmap, counts
  int32_t* mis_x_idx;
  uint32_t* mis_x_val;
  int32_t* mis_y_idx;
  uint32_t* mis_y_val;
  int32_t* mis_j_idx;
  int32_t* mis_ymin;
  uint32_t* mis_decided;
  int32_t* mis_cnt;
  void* mis_graph[SPMSPV_NUM_SCHEDULES / 2];
  // maximum bipartite matching (first use): frontier columns and the next
  // frontier, y (rows), row parents, column roots, the leaf row of each
  // root, visited rows, counts
  int32_t* mcm_x_idx;
  int32_t* mcm_x2_idx;
  int32_t* mcm_y_idx;
  uint32_t* mcm_y_val;
  int32_t* mcm_parent_r;
  int32_t* mcm_root_c;
  int32_t* mcm_leaf;
  uint32_t* mcm_visited;
  int32_t* mcm_cnt;
  void* mcm_graph[SPMSPV_NUM_SCHEDULES / 2];
  // presort of x (SPMSPV_SORT_X, first use): id bitmap (kept zero between
  // calls), parked values, the sorted x, look-back words + ticket
  uint32_t* sx_bits;
  uint32_t* sx_dense;
  int32_t* sx_idx;
  uint32_t* sx_val;
  unsigned long long* sx_status;
  int32_t* bfs_count;   // [4] device counters
};

namespace spmspv {
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* where);
int check_handle(const spmspv_handle* h);
Sched decode_schedule(const spmspv_handle* h, int id);
int run_push(spmspv_handle* h, int sem, const int32_t* x_idx, const uint32_t* x_val, int f,
             const int32_t* f_dev, const uint32_t* mask, int mask_comp, const Sched& sc,
             int32_t* y_idx, uint32_t* y_val, int32_t y_cap, int32_t* d_nnz_y, bool bfs,
             uint32_t* mask_update, cudaStream_t s);
// Returns -1 when the pull direction is not available for this handle/semiring.
// early_exit: (min, select2nd) with x(j) = j and ascending row ids: a row
// stops at its first frontier neighbour.
int run_pull_if_available(spmspv_handle* h, int sem, const int32_t* x_idx, const uint32_t* x_val,
                          int f, const uint32_t* mask, int mask_comp, const Sched& sc,
                          int32_t* y_idx, uint32_t* y_val, int32_t y_cap, int32_t* d_nnz_y,
                          cudaStream_t s, int early_exit = 0);
void release_extras(spmspv_handle* h);
void release_bfs_graphs(spmspv_handle* h);
void release_batch(spmspv_handle* h);
void release_k6(spmspv_handle* h);
void release_hostio(spmspv_handle* h);
void release_cc(spmspv_handle* h);
void release_mis(spmspv_handle* h);
void release_mcm(spmspv_handle* h);
// Sorts x by index into h->sx_idx / h->sx_val (sortx.cu); x_val may be NULL.
int sort_x(spmspv_handle* h, const int32_t* x_idx, const uint32_t* x_val, int32_t f, cudaStream_t s);
void release_sortx(spmspv_handle* h);
// Graph loops (graph_loop.cu).  build_while_graph captures `body` (given the
// loop's condition handle and the capture stream) as the body of a WHILE node
// whose condition starts at 1, and instantiates the graph.
int build_while_graph(spmspv_handle* h,
                      const std::function<int(cudaGraphConditionalHandle, cudaStream_t)>& body,
                      cudaGraphExec_t* out);
// One push SpMSpV inside a captured graph loop: x = (x_idx, x_val;
// x_val NULL gives x(j) = j) with its length read from f_dev on the device,
// rows whose bit is set in skip_rows produce nothing, y to (y_idx, y_val) with
// capacity m and its length in the device state.
int graph_spmspv(spmspv_handle* h, int sem, const Sched& sc, const int32_t* x_idx,
                 const uint32_t* x_val, const int32_t* f_dev, const uint32_t* skip_rows,
                 int32_t* y_idx, uint32_t* y_val, cudaStream_t s);
// The batched form as one persistent launch (batched_k6.cu); reads x_cnt on
// the host first (one synchronisation of `s`).  masks are complemented.
// x_ids: (min, select2nd) with every x value below INT32_MAX (vertex ids), so
// the merge may mark empty rows with INT32_MAX.
int run_batched_k6(spmspv_handle* h, int sem, int32_t B, const int32_t* x_off, const int32_t* x_cnt,
                   const int32_t* x_idx, const uint32_t* x_val, const uint32_t* masks, int64_t mask_stride,
                   uint32_t opts, const int32_t* y_off, const int32_t* y_cap, int32_t* y_idx, uint32_t* y_val,
                   int32_t* d_nnz_y, cudaStream_t s, bool x_ids = false);
// Reads and clears the status words of the batched lanes' workspaces (after
// the caller has synchronised the stream); CUDA errors are returned in *e.
uint32_t batch_collect_status(spmspv_handle* h, cudaError_t* e);
void release_tune(spmspv_handle* h);
// Autotuner (autotune.cu).  kind: 0 batched SpMSpV, 1 multi-source BFS, 2 ACL.
uint64_t tune_key(int kind, int sem, int masked, int32_t B, int64_t total_f);
// Runs `run(lanes, schedule opts)` with the cached choice for `key`, or times
// every candidate on `s` (each run twice, the second timed) and caches the best.
// Candidates by `forms`: kTuneLanes, lanes 2/4/8/16 x push schedules
// 0..nsched-1; kTunePersistent, the persistent form (lanes 0) x the schedules
// and lanes 4 and 16 x schedules 2 and 5; kTuneBoth, both full lists.
enum { kTuneLanes = 0, kTunePersistent = 1, kTuneBoth = 2 };
int tune_and_run(spmspv_handle* h, uint64_t key, cudaStream_t s,
                 const std::function<int(int32_t, uint32_t)>& run, int nsched = 6, int forms = kTuneLanes);
cudaError_t alloc_pull_buffers(spmspv_handle* h);
int pull_available(const spmspv_handle* h, int sem);
// BFS pull kernel of a batched lane (the lane's job names the source's arrays)
cudaError_t launch_pull_rows_lane(const spmspv_handle* sub, int early_exit, cudaStream_t s);
int ensure_bfs_buffers(spmspv_handle* h);
// The persistent BFS kernel of the adaptive schedules (bfs_fused.cu): its grid
// (every CTA resident; 0 if it cannot run) and its cooperative launch.
int fused_bfs_grid(const spmspv_handle* h);
cudaError_t launch_bfs_fused(const spmspv_handle* h, int grid, cudaStream_t s);
// Per-stage event recording (no-ops unless spmspv_profile_begin was called).
void prof_call_begin(spmspv_handle* h, cudaStream_t s);
void prof_mark(spmspv_handle* h, int stage, cudaStream_t s);
}  // namespace spmspv
