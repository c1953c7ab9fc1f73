// Internal declarations shared by the CUDA translation units of the library.
// Nothing here is part of the C ABI (include/spmspv.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "spmspv.h"

namespace spmspv {

// ---- semirings (same ids as the C ABI) ----
constexpr int kPlusTimes = SPMSPV_PLUS_TIMES_F32;
constexpr int kMinSelect2nd = SPMSPV_MIN_SELECT2ND_I32;
constexpr int kOrAnd = SPMSPV_OR_AND_BOOL;

// ---- K1: work estimation (prefix sum of selected column lengths) ----
constexpr int K1_THREADS = 256;
constexpr int K1_ITEMS = 8;
constexpr int K1_TILE = K1_THREADS * K1_ITEMS;  // x entries per scan tile

// ---- K2: expand + multiply + bucket scatter ----
// Tile starts are recorded every QF products; a K2 tile covers q = QF or
// 2*QF products (the "work quantum" of the schedule).
constexpr int QF = 2048;
constexpr int K2_THREADS = 512;
constexpr int K2_MIN_BLOCKS = 2;             // resident CTAs per SM the register budget allows
constexpr int K2_IMAX = 8;                   // products per thread at q = 4096
constexpr int QMAX = K2_THREADS * K2_IMAX;   // 4096

// ---- K3: per-bucket SPA merge + ordered compaction ----
constexpr int K3_THREADS = 512;

// ---- bucket row widths ----
constexpr int LWB_MIN = 7;    // 128 rows
constexpr int LWB_MAX = 15;   // 32768 rows (local row fits in uint16)
constexpr int NB_K2_MAX = 8192;   // buckets a K2 tile histograms in shared memory
// A BFS level whose products number at most this many runs in the direct
// form: K2 applies (min, select2nd) straight to the level and parent arrays
// with global atomics (the dense output arrays are the SPA) and K3 only
// closes the level; above it the bucketed form runs.
constexpr int32_t BFS_DIRECT_MAX = 1 << 21;
// A (+,*) product with at least PLUS_DIRECT_PER_ROW * m products (W) runs in
// the direct form when the handle has a dense y accumulator (m <= DIRECT_M_MAX):
// K2 adds every product into the accumulator in global memory (L2-resident
// at these sizes) and K3 reads the touched rows back in order, resetting
// them; below that W the bucketed form runs (measured crossover on R-MAT
// s20 and s22: between 0.7 m and 2.2 m products).
constexpr int PLUS_DIRECT_PER_ROW = 2;
constexpr int32_t DIRECT_M_MAX = 1 << 24;
constexpr int BFILL_STRIDE = 32;  // bucket fill counters sit 128 bytes apart (own L2 line)

// ---- hub ("hot") rows: the largest-degree rows, combined per K2 tile ----
constexpr int HOT_MAX = 1024;          // at most this many hot rows
constexpr int HOT_MIN_DEG = 512;       // a hot row has at least this many nonzeros


// ---- device status bits ----
constexpr uint32_t ST_CAPACITY = SPMSPV_DEV_CAPACITY;
constexpr uint32_t ST_TIMEOUT = SPMSPV_DEV_TIMEOUT;
constexpr uint32_t ST_BOUND = SPMSPV_DEV_BOUND;
constexpr uint32_t ST_INDEX = 4u;     // an x index or bucket fill was out of range

// Bounded waits: iterations of a spin (each with a short sleep) before a
// wait gives up and records ST_TIMEOUT.
constexpr uint32_t SPIN_LIMIT = 1u << 22;

// Look-back status word: flag in the two top bits.
constexpr unsigned long long LB_FLAG_AGG = 1ull << 62;
constexpr unsigned long long LB_FLAG_INC = 2ull << 62;
constexpr unsigned long long LB_FLAG_MASK = 3ull << 62;
constexpr unsigned long long LB_VAL_MASK = ~LB_FLAG_MASK;

// Per-call state kept on the device so that every launch has a fixed
// configuration and the host never waits for a count.
struct DevState {
  int32_t f;           // nnz(x) of the current call
  int32_t fc;          // x entries whose column is non-empty
  int32_t W;           // products: sum of the selected column lengths
  int32_t lwb;         // log2 bucket row width of this call
  int32_t q;           // work quantum (products per K2 tile)
  int32_t dir;         // 0 push (bucketed SpMSpV), 1 pull (masked SpMV)
  uint32_t status;     // sticky SPMSPV_DEV_* / ST_* bits
  int32_t nnz_y;       // size of y of the last call
  uint32_t k1_ticket;  // dynamic tile counter of K1
  uint32_t k3_ticket;  // dynamic bucket counter of K3
  int32_t maxdeg;      // largest selected column length (selector feature)
  int32_t sched;       // schedule id of the current call
  int32_t level;       // BFS level being discovered
  uint32_t pull_ticket;  // dynamic row-tile counter of the pull kernel
  int32_t nvisited;    // BFS: vertices reached so far
  int32_t maskcnt;     // rows with their mask bit set (selector feature)
  int32_t last_maxdeg;   // maxdeg and maskcnt of the last finished call
  int32_t last_maskcnt;
  int32_t* bfs_level;  // BFS outputs of the current search
  int32_t* bfs_parent;
  int32_t* cc_labels;  // connected components: the caller's labels
  int32_t* mis_in;     // maximal independent set: the caller's membership flags
  int32_t* mcm_mate_r;  // bipartite matching: the caller's mate arrays (rows, columns)
  int32_t* mcm_mate_c;
  uint32_t* bfs_fb;    // BFS: two frontier bitmaps of ceil(n/32) words; level L reads
                       // bitmap (L-1)&1 (pull) and writes bitmap L&1 (K3 or pull)
  uint32_t k1_done;    // K1 CTAs finished; the last one runs the selector (self-resetting)
  int32_t feat_dev;    // 1 when the current call's selector wrote feat[] (cleared by every K1)
  float feat[6];       // the six selector features as the device computed them
  int32_t bfs_acc;     // BFS level in the direct form: vertices found so far (reset by K1)
  int32_t* bfs_front;  // single-source BFS: the frontier list (x of a level, then its y)
  uint32_t fused_count;  // persistent BFS kernel: grid barrier arrivals (monotonic in a search)
  uint32_t fused_gen;    // persistent BFS kernel: barriers passed so far in the search
  int32_t fused_cnt[3];  // persistent BFS kernel, per level mod 3: vertices found,
  long long fused_w[4];  //   their products, non-empty columns and largest column; [3]: the
  int32_t fused_fc[4];   //   counts of the frontier a launch starts from (zeroed by K1)
  int32_t fused_md[4];
  long long edges_seen;  // BFS: column lengths summed over every frontier so far (the rule's m_u)
};

// Selector run inside the work scan by its last CTA to finish: weights (NULL:
// no selection in this launch), whether pull may be chosen, whether the mask
// is the BFS visited set (its population is then the visited count), and the
// conditional handles of a graph level (use_cond = 0 outside such graphs).
struct SelArgs {
  const float* w;
  int rule;          // 1: the direction-optimizing rule decides instead of the network
  int allow_pull;
  int bfs;
  int use_cond;
  int lwb_lo;
  int32_t direct_max;  // BFS: a level of at most this many products runs push (direct form)
  cudaGraphConditionalHandle c_push;
  cudaGraphConditionalHandle c_pull;
};

// One frontier of a batch, as the batched lanes hand it to the kernels
// (device memory; read at the start of K1, K2 and K3 when present).
struct Job {
  const int32_t* x_idx;
  const uint32_t* x_val;
  const uint32_t* mask;
  int32_t* y_idx;
  uint32_t* y_val;
  int32_t* d_nnz_y;
  int32_t* level;      // BFS mode: this source's outputs and visited bitmap
  int32_t* parent;
  uint32_t* visited;
  uint32_t* fb;        // BFS mode with the learned schedule: this source's two frontier
                       // bitmaps (level L reads bitmap (L-1)&1 and writes bitmap L&1)
  int32_t f;
  int32_t y_cap;
  int32_t b;           // frontier index, -1 when the queue was empty
  int32_t lvl;         // BFS mode: the level being discovered
  int32_t nvis;        // BFS mode: vertices this source has reached (selector feature)
};

struct Workspace {
  DevState* st;
  int32_t* cw;          // [n+1] exclusive work offsets of the compacted x entries
  int32_t* cb;          // [n]   first position of each compacted x entry's column
  uint32_t* cx;         // [n]   x value (32-bit payload) of each compacted entry
  int32_t* tile_k0;     // [nnz/QF + 2] compacted entry holding product t*QF
  unsigned long long* k1_status;  // [ceil(n/K1_TILE)] look-back words of K1
  int32_t* bfill;       // [nb_fine * BFILL_STRIDE] fill counters of the buckets
  unsigned long long* k3_status;  // [nb_fine] look-back words of K3
  int32_t* rbase;       // [nb_fine+1] first slot of each fine bucket's region
  uint16_t* brow;       // [nnz] bucket entries: row offset inside the bucket
  uint32_t* bval;       // [nnz] bucket entries: 32-bit value
  // hub rows (nhot of them, 0 when no row has HOT_MIN_DEG nonzeros)
  int nhot;
  const int32_t* hot_rows;   // [HOT_MAX] row ids, ascending
  const int32_t* hot_start;  // [nb_fine+1] first hot index of each fine bucket
  const int32_t* rowidx_k2;  // [nnz] row ids with hub row r replaced by m + its hub index
  unsigned long long* pull_status;  // [pull tiles] look-back words of the pull kernel
  int pull_tiles;
  const Job* job;            // batched lanes: the current frontier (NULL otherwise)
  uint32_t* hot_val;         // [HOT_MAX] per-call sums of the hot rows
  uint32_t* hot_touch;       // [HOT_MAX] 1 when a hot row received a product this call
  float* ydense;             // [m] dense (+,*) accumulator of the direct form, -0.0 in every
                             // row between calls (NULL when m > DIRECT_M_MAX)
};

// ---- pull direction (matrix-driven masked SpMV) ----
constexpr int PULL_THREADS = 256;
constexpr int PULL_ROWS = PULL_THREADS * 32;  // rows per pull tile: one 32-row word per thread

struct Matrix {
  int32_t m = 0, n = 0;
  int64_t nnz = 0;
  const int32_t* colptr = nullptr;  // CSC: [n+1] column pointers; DCSC: [nzc+1] pointers of the stored columns
  const int32_t* rowidx = nullptr;
  const float* val = nullptr;  // NULL for a pattern matrix
  // DCSC (Sec. II-C): only the nzc columns with a stored entry are kept, with
  // their ids in jc (ascending), plus an auxiliary index for constant
  // expected-time column lookup: aux[k] = the first position p with
  // jc[p] >= k << aux_shift.  jc == NULL for CSC.
  const int32_t* jc = nullptr;
  const int32_t* aux = nullptr;
  int32_t nzc = 0;
  int aux_shift = 0;
};

// [c0, c1) = the range of column j's entries in rowidx (empty when a DCSC
// matrix does not store column j): a binary search among the stored columns
// of j's aux chunk, which holds about one column on average.
__device__ __forceinline__ void col_range(const int32_t* __restrict__ colptr, const int32_t* __restrict__ jc,
                                          const int32_t* __restrict__ aux, int aux_shift, int32_t j,
                                          int32_t& c0, int32_t& c1) {
  if (!jc) {
    c0 = colptr[j];
    c1 = colptr[j + 1];
    return;
  }
  const int32_t k = j >> aux_shift;
  int32_t lo = aux[k];
  const int32_t end = aux[k + 1];
  int32_t hi = end;
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    if (jc[mid] < j) lo = mid + 1;
    else hi = mid;
  }
  if (lo < end && jc[lo] == j) {
    c0 = colptr[lo];
    c1 = colptr[lo + 1];
  } else {
    c0 = 0;
    c1 = 0;
  }
}

struct Sched {
  int id;    // schedule id: dir * 6 + quantum * 3 + width
  int dir;   // 0 push, 1 pull
  int q;     // QF or 2*QF
  int lwb;   // log2 bucket width
};

// Entries the work scan's compaction (cw, cb, cx) can hold: one per x entry
// whose column has an entry, so at most the number of stored columns.
inline int32_t compaction_capacity(const Matrix& A) {
  return A.jc ? (A.nzc < A.n ? A.nzc : A.n) : A.n;
}

// Launchers (kernels.cu).  All launches are asynchronous on `s`.
cudaError_t launch_k1(int sem, const Matrix& A, const Workspace& ws, int nb_fine,
                      const int32_t* x_idx, const uint32_t* x_val, int f, const int32_t* f_dev,
                      int grid, const Sched* forced, cudaStream_t s, const uint32_t* mask = nullptr,
                      const SelArgs* sel = nullptr);
cudaError_t launch_k1_bfs(const Matrix& A, const Workspace& ws, int nb_fine, const int32_t* x_idx,
                          const int32_t* f_dev, int grid, const Sched* sc, cudaStream_t s,
                          const uint32_t* mask, const SelArgs* sel = nullptr);
cudaError_t launch_row_degrees(const Matrix& A, int32_t* deg, int32_t* maxdeg, cudaStream_t s);
cudaError_t launch_rows_unsorted(const Matrix& A, int32_t* unsorted, cudaStream_t s);
cudaError_t launch_relabel_hubs(const Matrix& A, const int32_t* hub_of_row, int32_t* out,
                                cudaStream_t s);
// q_hint: the work quantum when the host knows it (selects a kernel compiled
// for it), 0 when the device picks it
// direct_max: a BFS level (the (min, select2nd) push of a search) runs in
// the direct form when its work is at most this many products; 0 for calls
// that are not BFS levels.  K2 and K3 of one level get the same value.
// use_cond/cond (BFS levels in a graph loop): K3 sets the loop's condition
// when it closes the level (another level while this one found vertices).
// plus_direct_min: a (+,*) call with at least this many products runs in the
// direct form (0: never); K2 and K3 of one call get the same value.
cudaError_t launch_k2(int sem, const Matrix& A, const Workspace& ws, int lwb_lo, int nb_fine,
                      const uint32_t* mask, int mask_comp, int grid, size_t smem, cudaStream_t s,
                      int only_push = 0, int q_hint = 0, int32_t direct_max = 0,
                      int32_t plus_direct_min = 0);
cudaError_t launch_k3(int sem, bool bfs, const Matrix& A, const Workspace& ws, int lwb_lo,
                      int nb_fine, int32_t* y_idx, uint32_t* y_val, int32_t y_cap, int32_t* d_nnz_y,
                      uint32_t* mask_update, int grid, size_t smem, cudaStream_t s,
                      int only_push = 0, int32_t direct_max = 0, int use_cond = 0,
                      cudaGraphConditionalHandle cond = 0, int32_t plus_direct_min = 0);
// Sets n 32-bit words to `value`.
cudaError_t launch_fill_u32(uint32_t* p, int64_t n, uint32_t value, cudaStream_t s);
cudaError_t launch_bucket_sizes(const Matrix& A, int lwb_lo, int nb_fine, int32_t* counts,
                                unsigned int* bad, cudaStream_t s);
// K2 shared memory: cb - cw and x value of the tile's x entries (whose bytes
// then hold the tile's staged (row, value) pairs), the bitmap of entry starts,
// the bucket histogram and slots (one more for the hub bucket), and the
// hub-row tables.
__host__ __device__ constexpr size_t k2_smem_bytes(int nb_fine, bool hot) {
  return sizeof(uint32_t) * (QMAX / 32) + sizeof(int32_t) * (QMAX + 1) +
         sizeof(uint32_t) * (QMAX + 1) + sizeof(int32_t) * ((size_t)nb_fine + 1) * 2 + 64 +
         (hot ? sizeof(uint32_t) * HOT_MAX * 2 + sizeof(uint32_t) * (HOT_MAX / 32) + 64 : 0);
}
// K3 shared memory: the SPA values and the occupancy bitmap of one bucket
// K3 shared memory: the SPA values and the occupancy bitmap of one bucket
__host__ __device__ constexpr size_t k3_smem_bytes(int lwb) {
  return ((size_t)1 << lwb) * sizeof(uint32_t) + (((size_t)1 << lwb) / 32) * sizeof(uint32_t);
}
constexpr size_t SMEM_PER_BLOCK_MAX = 227 * 1024;
static_assert(k2_smem_bytes(NB_K2_MAX, true) + 128 <= SMEM_PER_BLOCK_MAX, "K2 layout too large");
static_assert(k3_smem_bytes(LWB_MAX) + 4096 <= SMEM_PER_BLOCK_MAX, "K3 layout too large");
cudaError_t set_kernel_attributes(size_t k2_smem, size_t k3_smem_max);
int k3_blocks_per_sm(int sem, size_t smem);
int k2_blocks_per_sm(int sem, size_t smem);

}  // namespace spmspv
