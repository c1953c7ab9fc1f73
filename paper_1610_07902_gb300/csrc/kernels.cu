// SpMSpV kernels for sm_103a: y <- A (+).(x) x with A in CSC, x and y sparse.
//
// The three steps of Algorithm 1 (Sec. III) and the counting pre-pass of
// Algorithm 2, re-designed for one GB300:
//
//   K1 work_scan      Algorithm 2's role: instead of counting (thread, bucket)
//                     insertions, one decoupled-look-back prefix sum over the
//                     selected column lengths gives every product a global
//                     rank; x entries with an empty column are dropped and the
//                     first x entry of every QF-product tile is recorded
//                     (a merge-path split: every K2 tile then holds the same
//                     number of products, whatever the column lengths).
//   K2 expand_scatter Step 1: a tile of q products is gathered (coalesced
//                     loads of row ids and values), multiplied, optionally
//                     filtered by the mask, counted per row-range bucket in
//                     shared memory, staged bucket-by-bucket in shared memory
//                     and written to the buckets in runs; one global atomic
//                     per (tile, non-empty bucket) reserves each run.
//   K3 bucket_merge   Steps 2 and 3: a CTA owns one bucket at a time, merges
//                     it into a shared-memory SPA with the semiring's add,
//                     marks occupied rows in a bitmap, and writes its rows in
//                     ascending order at the offset given by a decoupled
//                     look-back over the buckets (the prefix sum of Step 3).
//
// Bucket b holds rows [b*Wb, (b+1)*Wb) with Wb a power of two; the paper's
// floor(i*nb/m) assignment is the same row-range split with nb = m/Wb.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "device_util.cuh"
#include "expand_dev.cuh"
#include "selector_dev.cuh"
#include "spmspv_internal.cuh"

namespace spmspv {

// ------------------------------------------------------------------------
// K1: work scan + compaction + tile starts
// ------------------------------------------------------------------------
__host__ __device__ constexpr int k1_pad(int e) { return e + (e >> 5); }
constexpr int K1_SMEM_WORDS = K1_TILE + K1_TILE / 32;

// Packed scan value: bits [0,31) = products, bits [31,62) = non-empty entries.
constexpr unsigned long long K1_CNT_ONE = 1ull << 31;
constexpr unsigned long long K1_SUM_MASK = (1ull << 31) - 1;

__global__ void __launch_bounds__(K1_THREADS)
k1_work_scan(const int32_t* x_idx, const uint32_t* x_val, int f_host, const int32_t* f_dev,
             const int32_t* __restrict__ colptr, const int32_t* __restrict__ jc,
             const int32_t* __restrict__ aux, int aux_shift, int32_t qcap, int32_t n,
             int64_t nnz, Workspace ws, int nb_fine, int sem, int forced, int f_dir, int f_q,
             int f_lwb, int bfs_level_inc, const uint32_t* __restrict__ mask, int32_t m,
             SelArgs sel) {
  __shared__ int32_t s_deg[K1_SMEM_WORDS];
  __shared__ int s_last;
  __shared__ int32_t s_c0[K1_SMEM_WORDS];
  __shared__ uint32_t s_xv[K1_SMEM_WORDS];
  __shared__ unsigned long long s_warp[K1_THREADS / 32 + 1];
  __shared__ unsigned long long s_prefix;
  __shared__ uint32_t s_tile;
  __shared__ int s_maxdeg;
  __shared__ int s_maskcnt;

  pdl_launch_next();  // the expand step may be scheduled now; it waits for this kernel
  DevState* st = ws.st;
  const int tid = threadIdx.x;
  const int bfs_mode = bfs_level_inc;  // a BFS level (single source or a batched lane's)
  if (ws.job) {  // a batched lane: this frontier's x
    x_idx = ws.job->x_idx;
    x_val = bfs_level_inc ? reinterpret_cast<const uint32_t*>(ws.job->x_idx) : ws.job->x_val;
    f_dev = &ws.job->f;
    bfs_level_inc = 0;
  }
  const int f = f_dev ? *f_dev : f_host;
  const uint32_t nt1 = (uint32_t)((f + K1_TILE - 1) / K1_TILE);

  if (blockIdx.x == 0) {
    // reset the state the later kernels of this call accumulate into
    for (int b = tid; b < nb_fine; b += K1_THREADS) {
      ws.bfill[(size_t)b * BFILL_STRIDE] = 0;
      ws.k3_status[b] = 0ull;
    }
    if (bfs_mode && ws.pull_status)
      for (int i = tid; i < ws.pull_tiles; i += K1_THREADS) ws.pull_status[i] = 0ull;
    const uint32_t hid = sem == kMinSelect2nd ? 0x7fffffffu : 0u;
    for (int h = tid; h < ws.nhot; h += K1_THREADS) {
      ws.hot_val[h] = hid;
      ws.hot_touch[h] = 0u;
    }
    if (tid == 0) {
      st->f = f;
      st->k3_ticket = 0u;
      st->feat_dev = 0;
      st->bfs_acc = 0;
      if (forced) {
        st->dir = f_dir;
        st->q = f_q;
        st->lwb = f_lwb;
        st->sched = forced - 1;
      }
      if (bfs_mode) {
        st->pull_ticket = 0u;  // the level may run the pull kernel
        st->fused_w[3] = 0;    // the persistent BFS kernel's next launch counts from zero
        st->fused_fc[3] = 0;
        st->fused_md[3] = 0;
      }
      if (bfs_level_inc) {
        // (an empty frontier only reaches here after the persistent kernel
        // of the learned schedule finished the search: no further level)
        if (f > 0) st->level += 1;
      } else if (!ws.job) {
        st->bfs_level = nullptr;  // not a BFS level
      }
      if (bfs_mode && ws.job) st->nvisited = ws.job->nvis;  // this source's, for the selector
      if (f == 0) {
        st->fc = 0;
        st->W = 0;
        ws.cw[0] = 0;
        ws.tile_k0[0] = 0;
      }
    }
  }
  // a CTA beyond the tiles has nothing to do unless it counts mask bits (the
  // others take every tile: the tickets are dynamic)
  if (blockIdx.x > 0 && blockIdx.x >= nt1 && !mask) return;
  if (tid == 0) {
    s_maxdeg = 0;
    s_maskcnt = 0;
  }

  int maxdeg = 0;
  uint32_t my_tiles = 0;
  for (;;) {
    if (tid == 0) s_tile = atomicAdd(&st->k1_ticket, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= nt1) break;
    ++my_tiles;
    const int64_t base = (int64_t)tile * K1_TILE;

    // striped, coalesced loads of x, then of the two column pointers of
    // every entry, all issued before any is used
    int32_t jj[K1_ITEMS];
    uint32_t xvv[K1_ITEMS];
#pragma unroll
    for (int i = 0; i < K1_ITEMS; ++i) {
      const int64_t k = base + i * K1_THREADS + tid;
      jj[i] = -1;
      xvv[i] = 0u;
      if (k < f) {
        jj[i] = x_idx[k];
        xvv[i] = x_val ? x_val[k] : 0u;
      }
    }
    int32_t c0v[K1_ITEMS], c1v[K1_ITEMS];
#pragma unroll
    for (int i = 0; i < K1_ITEMS; ++i) {
      c0v[i] = 0;
      c1v[i] = 0;
      const int64_t k = base + i * K1_THREADS + tid;
      if (k < f) {
        const int32_t j = jj[i];
        if (j >= 0 && j < n) {
          col_range(colptr, jc, aux, aux_shift, j, c0v[i], c1v[i]);
        } else {
          atomicOr(&st->status, ST_INDEX);
        }
        if (!x_val) xvv[i] = (uint32_t)j;
      }
    }
#pragma unroll
    for (int i = 0; i < K1_ITEMS; ++i) {
      const int e = i * K1_THREADS + tid;
      s_deg[k1_pad(e)] = c1v[i] - c0v[i];
      s_c0[k1_pad(e)] = c0v[i];
      s_xv[k1_pad(e)] = xvv[i];
    }
    __syncthreads();

    // blocked: thread owns entries [tid*8, tid*8+8) of the tile
    unsigned long long tsum = 0;
#pragma unroll
    for (int i = 0; i < K1_ITEMS; ++i) {
      const int d = s_deg[k1_pad(tid * K1_ITEMS + i)];
      tsum += (d > 0 ? K1_CNT_ONE : 0ull) + (unsigned long long)d;
      maxdeg = max(maxdeg, d);
    }
    unsigned long long btot;
    unsigned long long texcl = block_exclusive_sum<K1_THREADS>(tsum, s_warp, &btot);
    if (tid < 32) {
      const unsigned long long pre = warp_lookback(ws.k1_status, tile, btot, st);
      if (tid == 0) s_prefix = pre;
    }
    __syncthreads();
    unsigned long long run = s_prefix + texcl;
#pragma unroll
    for (int i = 0; i < K1_ITEMS; ++i) {
      const int e = tid * K1_ITEMS + i;
      const int d = s_deg[k1_pad(e)];
      if (d > 0) {
        const int32_t q = (int32_t)((run >> 31) & K1_SUM_MASK);
        const int32_t w = (int32_t)(run & K1_SUM_MASK);
        if (q < qcap && (int64_t)w + d <= nnz) {
          ws.cw[q] = w;
          ws.cb[q] = s_c0[k1_pad(e)];
          ws.cx[q] = s_xv[k1_pad(e)];
          for (int64_t t = ((int64_t)w + QF - 1) / QF; t * QF < (int64_t)w + d; ++t) ws.tile_k0[t] = q;
        } else {
          atomicOr(&st->status, ST_INDEX);  // more products than nonzeros: duplicate x indices
        }
        run += K1_CNT_ONE + (unsigned long long)d;
      }
    }
    if (tile == nt1 - 1 && tid == 0) {
      const unsigned long long tot = s_prefix + btot;
      int32_t fc = (int32_t)((tot >> 31) & K1_SUM_MASK);
      int32_t W = (int32_t)(tot & K1_SUM_MASK);
      if (fc > qcap || (int64_t)W > nnz) {  // only with duplicate x indices
        atomicOr(&st->status, ST_INDEX);
        fc = 0;
        W = 0;
      }
      st->fc = fc;
      st->W = W;
      ws.cw[fc] = W;
      ws.tile_k0[(W + QF - 1) / QF] = fc;
    }
    __syncthreads();
  }
  // selector features: degree statistics and the number of masked rows
  // one shared atomic per warp (all threads of the block share s_maxdeg)
  maxdeg = __reduce_max_sync(0xffffffffu, maxdeg);
  if ((tid & 31) == 0 && maxdeg > 0) atomicMax(&s_maxdeg, maxdeg);
  int32_t mc = 0;
  if (mask) {
    const int32_t words = (m + 31) / 32;
    for (int32_t i = blockIdx.x * K1_THREADS + tid; i < words; i += gridDim.x * K1_THREADS) {
      uint32_t wv = mask[i];
      if (i == words - 1 && (m & 31)) wv &= (1u << (m & 31)) - 1u;
      mc += __popc(wv);
    }
    mc = __reduce_add_sync(0xffffffffu, mc);
    if ((tid & 31) == 0 && mc) atomicAdd(&s_maskcnt, mc);
  }
  __syncthreads();
  if (tid == 0 && s_maxdeg > 0) atomicMax(&st->maxdeg, s_maxdeg);
  if (tid == 0 && s_maskcnt > 0) atomicAdd(&st->maskcnt, s_maskcnt);
  if (!sel.w && !sel.rule) return;
  // the selector runs in the CTA that finishes the last piece of work, once
  // every count is in: with a mask pass every CTA is a piece, otherwise every
  // tile plus block 0's state set-up (CTAs without a piece skip the counter)
  const uint32_t units = mask ? 1u : my_tiles + (blockIdx.x == 0 ? 1u : 0u);
  const uint32_t total = mask ? gridDim.x : nt1 + 1u;
  if (units == 0) return;
  if (tid == 0) {
    __threadfence();
    s_last = atomicAdd(&st->k1_done, units) + units == total;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    if (tid < 32) sel_choose_warp(sel.w, st, m, n, nnz, sel);  // (sel.rule: the rule instead)
    if (tid == 0) st->k1_done = 0u;
  }
}

cudaError_t launch_k1(int sem, const Matrix& A, const Workspace& ws, int nb_fine,
                      const int32_t* x_idx, const uint32_t* x_val, int f, const int32_t* f_dev,
                      int grid, const Sched* forced, cudaStream_t s, const uint32_t* mask,
                      const SelArgs* sel) {
  SelArgs none{};
  k1_work_scan<<<grid, K1_THREADS, 0, s>>>(x_idx, x_val, f, f_dev, A.colptr, A.jc, A.aux, A.aux_shift,
                                           compaction_capacity(A), A.n, A.nnz, ws, nb_fine,
                                           sem, forced ? forced->id + 1 : 0, forced ? forced->dir : 0,
                                           forced ? forced->q : 0, forced ? forced->lwb : 0, 0,
                                           mask, A.m, sel ? *sel : none);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------
// K2: expand + multiply + bucket scatter
// ------------------------------------------------------------------------

// One tile = q consecutive products (a merge-path slice of the selected
// columns).  Each warp takes a contiguous chunk of 32*items products with
// its lanes on consecutive products (coalesced row-id and value loads).  The
// x entry of a product comes from a bitmap of the tile's entry starts: the
// 32 products of one warp load are one bitmap word, so a lane's entry is the
// count of starts before its word plus a popcount inside the word (no
// search, no divergence).  Products are counted per bucket with
// shared-memory atomics, one warp scans the counts, every non-empty bucket
// gets one run reserved with a global atomic, the products are staged in
// shared memory grouped by bucket (in the bytes that held the tile's x
// entries) and written out in runs.  Hub rows (row ids >= m in the
// relabelled row-id array) are one more bucket of the histogram, the last:
// they are staged like the others and then summed into a per-CTA table in
// shared memory that is flushed once, when the CTA has no tile left, so a
// hub product costs what any product costs and no warp branches on it.
// IT: products per thread when the host knows the work quantum (4 or 8),
// 0 when the device decides it; MASKED: a mask may be given.

// Bucket of a product row id: its row range, the hub bucket nb, or -1 for
// "no product" and for an id outside [0, m) that is not a hub label (which
// only a matrix that was never checked at create can hold).
__device__ __forceinline__ int k2_bucket(uint32_t row, int32_t m, int nhot, int lwb, int nb) {
  if (row < (uint32_t)m) return (int)(row >> lwb);
  if (row - (uint32_t)m < (uint32_t)nhot) return nb;
  return -1;
}

// A BFS level in the direct form (few products): for every product (row i,
// frontier vertex j) with i unreached before this level, parent[i] =
// min(parent[i], j), and level[i] = L for the first product that finds i
// (compare-and-swap), which also appends i to the next frontier and sets its
// visited bit.  The parent array is the SPA: it holds -1 (as unsigned, the
// largest value) for every vertex not reached yet, so an unsigned min needs
// no initialisation of its own.  "Unreached before this level" is read from
// the level array (-1, or L when another product found i in this level), so
// the visited bits set during the level change nothing and the minimum is
// exact.  Every item's loads and atomics are issued before any result is
// used; one global atomic per warp and tile reserves the frontier slots.
// With the learned schedule this level's frontier bitmap is cleared here and
// K3 sets it (a later pull level reads it).
template <int IT>
__device__ void k2_bfs_direct(const int32_t* __restrict__ rowidx, Workspace ws, int32_t m, int64_t nnz,
                              uint32_t* __restrict__ visited, unsigned char* smem_raw) {
  const DevState* st = ws.st;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int32_t W = st->W, fc = st->fc, q = st->q;
  const int items = IT ? IT : q / K2_THREADS;
  const int ntiles = (int)(((int64_t)W + q - 1) / q);
  const int nhot = ws.nhot;
  const Job* job = ws.job;
  const int32_t L = job ? job->lvl : st->level;
  int32_t* level = job ? job->level : st->bfs_level;
  uint32_t* parent = reinterpret_cast<uint32_t*>(job ? job->parent : st->bfs_parent);
  int32_t* front = job ? job->y_idx : st->bfs_front;
  int32_t* acc = &ws.st->bfs_acc;
  uint32_t* fb = job ? job->fb : st->bfs_fb;
  if (fb) {  // this level's frontier bitmap, set again by K3
    const int64_t words = ((int64_t)m + 31) / 32;
    fb += (L & 1) ? words : 0;
    for (int64_t w = (int64_t)blockIdx.x * K2_THREADS + tid; w < words; w += (int64_t)gridDim.x * K2_THREADS)
      fb[w] = 0u;
  }
  if ((int)blockIdx.x >= ntiles) return;  // no tile for this CTA (tiles go round-robin)
  unsigned char* p = smem_raw;
  int32_t* kbase = (int32_t*)p; p += sizeof(int32_t) * (QMAX + 1);
  uint32_t* kx = (uint32_t*)p; p += sizeof(uint32_t) * (QMAX + 1);
  uint32_t* hbits = (uint32_t*)p; p += sizeof(uint32_t) * (QMAX / 32);
  int32_t* hrow = (int32_t*)p;  // hub row ids
  for (int i = tid; i < nhot; i += K2_THREADS) hrow[i] = ws.hot_rows[i];
  for (int i = tid; i < QMAX / 32; i += K2_THREADS) hbits[i] = 0u;
  __syncthreads();
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int32_t p0 = t * q;
    const int32_t np = min(q, W - p0);
    const int32_t k0 = ws.tile_k0[p0 / QF];
    const int32_t kend = (p0 + np == W) ? fc : ws.tile_k0[(p0 + np) / QF] + 1;
    const int32_t nk = max(1, min(kend - k0, QMAX + 1));
    for (int l = tid; l < nk; l += K2_THREADS) {
      const int32_t w = ws.cw[k0 + l];
      kbase[l] = ws.cb[k0 + l] - w;
      kx[l] = ws.cx[k0 + l];
      const int32_t off = w - p0;
      if (l > 0 && off > 0 && off < np) atomicOr(&hbits[off >> 5], 1u << (off & 31));
    }
    __syncthreads();
    uint32_t rrow[K2_IMAX], rval[K2_IMAX];
    if (np == items * K2_THREADS)
      k2_gather<kMinSelect2nd, IT, true>(rowidx, nullptr, hbits, kbase, kx, items, warp, lane, p0, np, nnz,
                                         rrow, rval);
    else
      k2_gather<kMinSelect2nd, IT, false>(rowidx, nullptr, hbits, kbase, kx, items, warp, lane, p0, np, nnz,
                                          rrow, rval);
    // the row of every item (hub labels mapped back), then its level
    int32_t lv[K2_IMAX];
#pragma unroll
    for (int i = 0; i < K2_IMAX; ++i) {
      uint32_t row = rrow[i];
      if (row != 0xffffffffu && row >= (uint32_t)m) {
        if (row - (uint32_t)m < (uint32_t)nhot) {
          row = (uint32_t)hrow[row - (uint32_t)m];
        } else {
          atomicOr(&ws.st->status, ST_INDEX);  // a row id outside [0, m): dropped, flagged
          row = 0xffffffffu;
        }
      }
      rrow[i] = row;
      lv[i] = row != 0xffffffffu ? __ldcg(level + row) : 0;
    }
    // the semiring's add on the dense parent array, then the first finder
    uint32_t found = 0u;
#pragma unroll
    for (int i = 0; i < K2_IMAX; ++i) {
      if (rrow[i] == 0xffffffffu || (lv[i] != -1 && lv[i] != L)) continue;
      atomicMin(parent + rrow[i], rval[i]);
      if (lv[i] == -1 && atomicCAS(level + rrow[i], -1, L) == -1) found |= 1u << i;
    }
    // one frontier reservation per warp, then the new vertices
    const int32_t c = __popc(found);
    int32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    int32_t base = 0;
    if (lane == 31 && incl > 0) base = atomicAdd(acc, incl);
    base = __shfl_sync(0xffffffffu, base, 31) + incl - c;
#pragma unroll
    for (int i = 0; i < K2_IMAX; ++i) {
      if (!((found >> i) & 1u)) continue;
      const uint32_t r = rrow[i];
      front[base++] = (int32_t)r;
      atomicOr(visited + (r >> 5), 1u << (r & 31));
    }
    __syncthreads();  // the entries of the next tile overwrite this one's
    for (int j = tid; j < QMAX / 32; j += K2_THREADS) hbits[j] = 0u;
    __syncthreads();
  }
}

// A (+,*) call in the direct form (many products): every product is added
// into the dense accumulator ws.ydense in global memory with a reduction
// (no result read back), after the mask.  Hub rows (ids >= m in the
// relabelled row-id array) are summed per CTA in shared memory first and
// added once, when the CTA has no tile left, so the most contended rows see
// one global add per CTA.  Rows keep -0.0 until touched (K2 stores +0.0 for
// a -0.0 product and -0.0 + p == p), so K3 finds them without a bitmap.
template <int IT, bool MASKED>
__device__ void k2_plus_direct(const int32_t* __restrict__ rowidx, const float* __restrict__ val, Workspace ws,
                               int32_t m, int64_t nnz, const uint32_t* mask, int mask_comp,
                               unsigned char* smem_raw) {
  const DevState* st = ws.st;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int32_t W = st->W, fc = st->fc, q = st->q;
  const int items = IT ? IT : q / K2_THREADS;
  const int ntiles = (int)(((int64_t)W + q - 1) / q);
  const int nhot = ws.nhot;
  float* yd = ws.ydense;
  if ((int)blockIdx.x >= ntiles) return;  // no tile for this CTA (tiles go round-robin)
  unsigned char* p = smem_raw;
  int32_t* kbase = (int32_t*)p; p += sizeof(int32_t) * (QMAX + 1);
  uint32_t* kx = (uint32_t*)p; p += sizeof(uint32_t) * (QMAX + 1);
  uint32_t* hbits = (uint32_t*)p; p += sizeof(uint32_t) * (QMAX / 32);
  uint32_t* hacc = (uint32_t*)p;              // hub sums of this CTA
  int32_t* hrow = (int32_t*)(hacc + HOT_MAX);  // hub row ids
  uint32_t* htb = (uint32_t*)(hrow + HOT_MAX); // hub touched bits
  if (nhot > 0) {
    for (int i = tid; i < HOT_MAX; i += K2_THREADS) {
      hacc[i] = 0u;
      hrow[i] = i < nhot ? ws.hot_rows[i] : 0;
    }
    for (int i = tid; i < HOT_MAX / 32; i += K2_THREADS) htb[i] = 0u;
  }
  for (int i = tid; i < QMAX / 32; i += K2_THREADS) hbits[i] = 0u;
  __syncthreads();
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int32_t p0 = t * q;
    const int32_t np = min(q, W - p0);
    const int32_t k0 = ws.tile_k0[p0 / QF];
    const int32_t kend = (p0 + np == W) ? fc : ws.tile_k0[(p0 + np) / QF] + 1;
    const int32_t nk = max(1, min(kend - k0, QMAX + 1));
    for (int l = tid; l < nk; l += K2_THREADS) {
      const int32_t w = ws.cw[k0 + l];
      kbase[l] = ws.cb[k0 + l] - w;
      kx[l] = ws.cx[k0 + l];
      const int32_t off = w - p0;
      if (l > 0 && off > 0 && off < np) atomicOr(&hbits[off >> 5], 1u << (off & 31));
    }
    __syncthreads();
    uint32_t rrow[K2_IMAX], rval[K2_IMAX];
    if (np == items * K2_THREADS)
      k2_gather<kPlusTimes, IT, true>(rowidx, val, hbits, kbase, kx, items, warp, lane, p0, np, nnz, rrow, rval);
    else
      k2_gather<kPlusTimes, IT, false>(rowidx, val, hbits, kbase, kx, items, warp, lane, p0, np, nnz, rrow, rval);
#pragma unroll
    for (int i = 0; i < K2_IMAX; ++i) {
      const uint32_t row = rrow[i];
      if (row == 0xffffffffu) continue;
      uint32_t r = row;
      int hs = -1;
      if (row >= (uint32_t)m) {
        if (row - (uint32_t)m >= (uint32_t)nhot) {
          atomicOr(&ws.st->status, ST_INDEX);  // a row id outside [0, m): dropped, flagged
          continue;
        }
        hs = (int)(row - (uint32_t)m);
        r = (uint32_t)hrow[hs];
      }
      if (MASKED && mask) {
        const uint32_t bit = (__ldg(mask + (r >> 5)) >> (r & 31)) & 1u;
        if (mask_comp ? bit != 0u : bit == 0u) continue;
      }
      if (hs >= 0) {
        spa_apply<kPlusTimes>(hacc, (uint32_t)hs, rval[i]);
        const uint32_t hb = 1u << (hs & 31);
        if (!(htb[hs >> 5] & hb)) atomicOr(&htb[hs >> 5], hb);
      } else {
        atomicAdd(yd + r, __uint_as_float(rval[i]));
      }
    }
    __syncthreads();  // the entries of the next tile overwrite this one's
    for (int j = tid; j < QMAX / 32; j += K2_THREADS) hbits[j] = 0u;
    __syncthreads();
  }
  if (nhot > 0) {
    for (int hs = tid; hs < nhot; hs += K2_THREADS)
      if ((htb[hs >> 5] >> (hs & 31)) & 1u) atomicAdd(yd + hrow[hs], __uint_as_float(hacc[hs]));
  }
}

template <int SEM, int IT, bool MASKED>
__global__ void __launch_bounds__(K2_THREADS, K2_MIN_BLOCKS)
k2_expand_scatter(const int32_t* __restrict__ rowidx, const float* __restrict__ val, Workspace ws,
                  int lwb_lo, int nb_fine, int32_t m, int64_t nnz, const uint32_t* mask,
                  int mask_comp, int only_push, int32_t direct_max, int32_t plus_direct_min) {
  pdl_wait();         // the work scan's outputs are complete and visible
  pdl_launch_next();  // the merge step may be scheduled now; it waits for this kernel
  if (only_push && ws.st->dir != 0) return;  // this call runs the pull direction
  if (ws.job) mask = ws.job->mask;
  extern __shared__ __align__(16) unsigned char k2_smem_raw[];
  if (SEM == kMinSelect2nd && MASKED && direct_max > 0 && ws.st->W <= direct_max) {
    if (!ws.job || ws.job->b >= 0)
      k2_bfs_direct<IT>(rowidx, ws, m, nnz, const_cast<uint32_t*>(mask), k2_smem_raw);
    return;
  }
  if (SEM == kPlusTimes && plus_direct_min > 0 && ws.st->W >= plus_direct_min) {
    k2_plus_direct<IT, MASKED>(rowidx, val, ws, m, nnz, mask, mask_comp, k2_smem_raw);
    return;
  }
  __shared__ int32_t s_kept, s_kept_n;

  unsigned char* p = k2_smem_raw;
  // the staged products of a tile share their bytes with the tile's x entries
  // (the entries are no longer read once the products are counted)
  uint2* stage = (uint2*)p;
  int32_t* kbase = (int32_t*)p; p += sizeof(int32_t) * (QMAX + 1);
  uint32_t* kx = (uint32_t*)p; p += sizeof(uint32_t) * (QMAX + 1);
  uint32_t* hbits = (uint32_t*)p; p += sizeof(uint32_t) * (QMAX / 32);  // entry starts of the tile
  int32_t* hist = (int32_t*)p; p += sizeof(int32_t) * (nb_fine + 1);  // counts, then stage offsets
  int32_t* gd = (int32_t*)p; p += sizeof(int32_t) * (nb_fine + 1);    // counts, then slot - stage offset
  uint32_t* hacc = (uint32_t*)p;                                      // hub sums of this CTA
  int32_t* hrow = (int32_t*)(hacc + HOT_MAX);                         // hub row ids
  uint32_t* htb = (uint32_t*)(hrow + HOT_MAX);                        // hub touched bits

  const DevState* st = ws.st;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int32_t W = st->W, fc = st->fc, q = st->q, lwb = st->lwb;
  const int sh = lwb - lwb_lo;
  const int nb = (int)(((int64_t)m + (1 << lwb) - 1) >> lwb);
  const uint32_t wmask = (1u << lwb) - 1u;
  const int items = IT ? IT : q / K2_THREADS;
  const int ntiles = (int)(((int64_t)W + q - 1) / q);
  const uint32_t ident = sr_identity<SEM>();
  const int nhot = ws.nhot;
  if ((int)blockIdx.x >= ntiles) return;  // no tile for this CTA (tiles go round-robin)

  if (nhot > 0) {
    for (int i = tid; i < HOT_MAX; i += K2_THREADS) {
      hacc[i] = ident;
      if (MASKED) hrow[i] = ws.hot_rows[i];
    }
    for (int i = tid; i < HOT_MAX / 32; i += K2_THREADS) htb[i] = 0u;
  }
  for (int i = tid; i < QMAX / 32; i += K2_THREADS) hbits[i] = 0u;
  __syncthreads();

  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int32_t p0 = t * q;
    const int32_t np = min(q, W - p0);
    const int32_t k0 = ws.tile_k0[p0 / QF];
    const int32_t kend = (p0 + np == W) ? fc : ws.tile_k0[(p0 + np) / QF] + 1;
    const int32_t nk = max(1, min(kend - k0, QMAX + 1));

    // the first K2_THREADS entries of every tile but a CTA's first were
    // loaded during the previous tile (below)
    for (int l = tid + (t != (int)blockIdx.x ? K2_THREADS : 0); l < nk; l += K2_THREADS) {
      const int32_t k = k0 + l;
      const int32_t w = ws.cw[k];
      kbase[l] = ws.cb[k] - w;
      kx[l] = ws.cx[k];
      const int32_t off = w - p0;  // entries after the first start inside the tile
      if (l > 0 && off > 0 && off < np) atomicOr(&hbits[off >> 5], 1u << (off & 31));
    }
    for (int b = tid; b <= nb; b += K2_THREADS) hist[b] = 0;
    __syncthreads();

    // ---- gather, multiply, filter, count per bucket ----
    uint32_t rrow[K2_IMAX], rval[K2_IMAX];
    int32_t rank[K2_IMAX];
    if (np == items * K2_THREADS)  // every item of every warp holds a product
      k2_gather<SEM, IT, true>(rowidx, val, hbits, kbase, kx, items, warp, lane, p0, np, nnz, rrow, rval);
    else
      k2_gather<SEM, IT, false>(rowidx, val, hbits, kbase, kx, items, warp, lane, p0, np, nnz, rrow, rval);
    const uint32_t mbits = (MASKED && mask) ? k2_mask_bits(mask, rrow, (uint32_t)m, (uint32_t)nhot, hrow) : 0u;
#pragma unroll
    for (int i = 0; i < K2_IMAX; ++i) {
      rank[i] = -1;
      const uint32_t row = rrow[i];
      const int b = k2_bucket(row, m, nhot, lwb, nb);
      if (b < 0) {
        if (row != 0xffffffffu) atomicOr(&ws.st->status, ST_INDEX);  // dropped, flagged
        continue;
      }
      bool keep = true;
      if (MASKED && mask) {
        const uint32_t bit = (mbits >> i) & 1u;
        keep = mask_comp ? (bit == 0u) : (bit != 0u);
      }
      if (keep) rank[i] = atomicAdd(&hist[b], 1);
    }
    __syncthreads();
    for (int j = tid; j < QMAX / 32; j += K2_THREADS) hbits[j] = 0u;  // the gather is done

    // ---- the next tile's x entries: in flight during this tile's scan,
    // reservation and stores, written to shared memory before the write-out ----
    const int tn = t + (int)gridDim.x;
    int32_t p0n = 0, npn = 0, nkn = 0, pw = 0, pcb = 0;
    uint32_t pcx = 0u;
    if (tn < ntiles) {
      p0n = tn * q;
      npn = min(q, W - p0n);
      const int32_t k0n = ws.tile_k0[p0n / QF];
      const int32_t kendn = (p0n + npn == W) ? fc : ws.tile_k0[(p0n + npn) / QF] + 1;
      nkn = max(1, min(kendn - k0n, QMAX + 1));
      if (tid < nkn) {
        pw = ws.cw[k0n + tid];
        pcb = ws.cb[k0n + tid];
        pcx = ws.cx[k0n + tid];
      }
    }

    // ---- one warp scans the bucket counts (the hub bucket last) ----
    if (warp == 0) {
      const int nbh = nb + 1;
      const int per = (nbh + 31) >> 5;
      const int b0 = lane * per, b1 = min(b0 + per, nbh);
      int32_t sum = 0;
      for (int b = b0; b < b1; ++b) sum += hist[b];
      int32_t x = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      int32_t run = x - sum;
      if (lane == 31) s_kept = x;
      for (int b = b0; b < b1; ++b) {
        const int32_t c = hist[b];
        if (b == nb) s_kept_n = run;
        gd[b] = c;
        hist[b] = run;
        run += c;
      }
    }
    __syncthreads();
    // ---- reserve one run per non-empty bucket (all threads) ----
    for (int b = tid; b < nb; b += K2_THREADS) {
      const int32_t c = gd[b];
      if (c > 0) {
        const int32_t base = ws.rbase[b << sh];
        const int32_t cap = ws.rbase[min((b + 1) << sh, nb_fine)] - base;
        const int32_t g = atomicAdd(&ws.bfill[(size_t)b * BFILL_STRIDE], c);
        if (g + c <= cap) {
          gd[b] = base + g - hist[b];
        } else {
          gd[b] = INT32_MIN;  // only reachable with duplicate x indices
          atomicOr(&ws.st->status, ST_INDEX);
        }
      }
    }
    // ---- stage the products grouped by bucket ----
#pragma unroll
    for (int i = 0; i < K2_IMAX; ++i)
      if (rank[i] >= 0)
        stage[hist[k2_bucket(rrow[i], m, nhot, lwb, nb)] + rank[i]] = make_uint2(rrow[i], rval[i]);
    __syncthreads();
    // ---- write the runs to the buckets; sum the hub products ----
    const int32_t kept_n = s_kept_n, kept = s_kept;
    for (int32_t s = tid; s < kept; s += K2_THREADS) {
      const uint2 e = stage[s];
      if (s < kept_n) {
        const int32_t g = gd[e.x >> lwb];
        if (g == INT32_MIN) continue;
        const int32_t dst = g + s;
        ws.brow[dst] = (uint16_t)(e.x & wmask);
        if (SEM != kOrAnd) ws.bval[dst] = e.y;
      } else {
        const uint32_t hs = e.x - (uint32_t)m;
        spa_apply<SEM>(hacc, hs, e.y);
        const uint32_t bit = 1u << (hs & 31);
        if (!(htb[hs >> 5] & bit)) atomicOr(&htb[hs >> 5], bit);
      }
    }
    __syncthreads();  // the staged products are written out: their bytes take the next entries
    if (tid < nkn) {  // the next tile's first entries (loaded during this tile)
      kbase[tid] = pcb - pw;
      kx[tid] = pcx;
      const int32_t off = pw - p0n;
      if (tid > 0 && off > 0 && off < npn) atomicOr(&hbits[off >> 5], 1u << (off & 31));
    }
  }
  // ---- the CTA's hub sums, once ----
  if (nhot > 0) {
    __syncthreads();
    for (int hs = tid; hs < nhot; hs += K2_THREADS) {
      if ((htb[hs >> 5] >> (hs & 31)) & 1u) {
        if (SEM == kPlusTimes)
          atomicAdd(reinterpret_cast<float*>(ws.hot_val + hs), __uint_as_float(hacc[hs]));
        else if (SEM == kMinSelect2nd)
          atomicMin(reinterpret_cast<int*>(ws.hot_val + hs), (int)hacc[hs]);
        ws.hot_touch[hs] = 1u;
      }
    }
  }
}

// The expand and merge steps follow the step before them with programmatic
// dependent launch when the stream is not being captured (graph loops keep
// plain launches): their CTAs are scheduled while the step before drains
// and wait in pdl_wait() for its results.
static bool pdl_allowed(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cs == cudaStreamCaptureStatusNone;
}

template <typename... KArgs, typename... Args>
static void launch_after(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s, bool pdl,
                         Args... args) {
  if (!pdl) {
    kernel<<<grid, block, smem, s>>>(args...);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <int SEM>
static void k2_variant(int it, bool masked, int grid, size_t smem, cudaStream_t s, const int32_t* rows,
                       const float* val, const Workspace& ws, int lwb_lo, int nb_fine, const Matrix& A,
                       const uint32_t* mask, int mask_comp, int only_push, int32_t direct_max,
                       int32_t plus_direct_min) {
  const bool pdl = pdl_allowed(s);
#define K2_GO(I, M)                                                                                       \
  launch_after(k2_expand_scatter<SEM, I, M>, grid, K2_THREADS, smem, s, pdl, rows, val, ws, lwb_lo, nb_fine, \
               A.m, A.nnz, mask, mask_comp, only_push, direct_max, plus_direct_min)
  constexpr int I1 = K2_IMAX, I2 = K2_IMAX / 2;
  if (masked) {
    if (it == I1) K2_GO(I1, true); else if (it == I2) K2_GO(I2, true); else K2_GO(0, true);
  } else {
    if (it == I1) K2_GO(I1, false); else if (it == I2) K2_GO(I2, false); else K2_GO(0, false);
  }
#undef K2_GO
}

cudaError_t launch_k2(int sem, const Matrix& A, const Workspace& ws, int lwb_lo, int nb_fine,
                      const uint32_t* mask, int mask_comp, int grid, size_t smem, cudaStream_t s,
                      int only_push, int q_hint, int32_t direct_max, int32_t plus_direct_min) {
  if (!ws.ydense) plus_direct_min = 0;
  const int32_t* rows = ws.nhot > 0 ? ws.rowidx_k2 : A.rowidx;
  // the batched lanes take their masks from the job: compile the mask path in
  const bool masked = mask != nullptr || ws.job != nullptr;
  const int it = q_hint == K2_IMAX * K2_THREADS ? K2_IMAX : q_hint == (K2_IMAX / 2) * K2_THREADS ? K2_IMAX / 2 : 0;
  switch (sem) {
    case kPlusTimes:
      k2_variant<kPlusTimes>(it, masked, grid, smem, s, rows, A.val, ws, lwb_lo, nb_fine, A, mask,
                             mask_comp, only_push, 0, plus_direct_min);
      break;
    case kMinSelect2nd:
      k2_variant<kMinSelect2nd>(it, masked, grid, smem, s, rows, nullptr, ws, lwb_lo, nb_fine, A, mask,
                                mask_comp, only_push, masked ? direct_max : 0, 0);
      break;
    default:
      k2_variant<kOrAnd>(it, masked, grid, smem, s, rows, nullptr, ws, lwb_lo, nb_fine, A, mask,
                         mask_comp, only_push, 0, 0);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------------
// K3: per-bucket SPA merge + ordered compaction (+ BFS update)
// ------------------------------------------------------------------------
// Two merge forms, chosen per bucket (the choice is uniform in the CTA):
//   dense   (many entries): every SPA slot starts at an "empty" value that no
//           merge can produce, so the semiring's add is the only shared-memory
//           update per entry and the occupied rows are read back from the SPA
//           itself.  (+,*): empty = -0.0f (K2 stores +0.0 for a -0.0 product,
//           and -0.0 + p == p, so a touched row never holds -0.0);
//           (min,select2nd) in BFS: empty = INT32_MAX (x values are vertex ids).
//           The compaction walks the SPA 32 rows per warp step (ballot).
//   sparse  (few entries, or no free empty value): an occupancy bitmap next to
//           the SPA, partially initialised (Sec. II-F), compacted per word.
constexpr int K3_WARPS = K3_THREADS / 32;
constexpr int K3_DENSE_MIN_WB = 32 * K3_WARPS;  // every warp walks whole 32-row words
constexpr int K3_DENSE_DIV = 8;                 // dense when entries >= rows / 8


// The end of a BFS level that K2 ran in the direct form: the level's count,
// the per-call state the work scan starts from, and (when a later level may
// pull) the new frontier's bits in this level's frontier bitmap.
__device__ void k3_bfs_direct_close(Workspace ws, int32_t m, const int32_t* y_idx, int32_t* d_nnz_y,
                                    int use_cond, cudaGraphConditionalHandle cond) {
  DevState* st = ws.st;
  const int tid = threadIdx.x;
  const int32_t total = st->bfs_acc;
  if (blockIdx.x == 0) {
    if (tid == 0) {
      if (use_cond) cudaGraphSetConditional(cond, (total > 0 && st->level <= m) ? 1u : 0u);
      st->k1_ticket = 0u;
      st->last_maxdeg = st->maxdeg;
      st->last_maskcnt = st->maskcnt;
      st->maxdeg = 0;
      st->maskcnt = 0;
      st->nnz_y = total;
      st->nvisited += total;
      if (d_nnz_y) *d_nnz_y = total;
    }
    const int nt1 = (st->f + K1_TILE - 1) / K1_TILE;
    for (int i = tid; i < nt1; i += K3_THREADS) ws.k1_status[i] = 0ull;
  }
  const int32_t lvl = ws.job ? ws.job->lvl : st->level;
  uint32_t* fb = ws.job ? ws.job->fb : st->bfs_fb;
  if (!fb) return;
  fb += (lvl & 1) ? ((int64_t)m + 31) / 32 : 0;
  for (int32_t k = blockIdx.x * K3_THREADS + tid; k < total; k += gridDim.x * K3_THREADS) {
    const int32_t r = y_idx[k];
    atomicOr(fb + (r >> 5), 1u << (r & 31));
  }
}

// The end of a (+,*) call in the direct form: the touched rows of the dense
// accumulator (those not holding -0.0), in ascending order, to y, each reset
// to -0.0 as it is read.  CTAs take row tiles of K3D_ROWS rows in ticket
// order; each warp reads its K3D_STEPS 32-row words of a tile at once
// (coalesced, kept in registers), ballots them, and a block scan plus a
// look-back over the tiles give each tile's offset in y.
constexpr int K3D_STEPS = 16;                          // 32-row words per warp and tile
constexpr int K3D_ROWS = K3_THREADS * K3D_STEPS;      // rows per tile (8192)

__device__ void k3_plus_direct(Workspace ws, int32_t m, int32_t* y_idx, uint32_t* y_val, int32_t y_cap,
                               int32_t* d_nnz_y) {
  DevState* st = ws.st;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ int32_t s_scan[K3_THREADS / 32 + 1];
  __shared__ uint32_t s_tk;
  __shared__ unsigned long long s_off;
  uint32_t* yd = reinterpret_cast<uint32_t*>(ws.ydense);
  constexpr uint32_t kEmpty = 0x80000000u;  // -0.0f
  if (blockIdx.x == 0) {
    if (tid == 0) {
      st->k1_ticket = 0u;
      st->last_maxdeg = st->maxdeg;
      st->last_maskcnt = st->maskcnt;
      st->maxdeg = 0;
      st->maskcnt = 0;
    }
    const int nt1 = (st->f + K1_TILE - 1) / K1_TILE;
    for (int i = tid; i < nt1; i += K3_THREADS) ws.k1_status[i] = 0ull;
  }
  const uint32_t ntiles = (uint32_t)(((int64_t)m + K3D_ROWS - 1) / K3D_ROWS);
  const uint32_t lt = (1u << lane) - 1u;
  for (;;) {
    if (tid == 0) s_tk = atomicAdd(&st->k3_ticket, 1u);
    __syncthreads();
    const uint32_t t = s_tk;
    if (t >= ntiles) break;
    const int64_t r0 = (int64_t)t * K3D_ROWS + (int64_t)warp * (K3D_STEPS * 32) + lane;
    uint32_t v[K3D_STEPS];
#pragma unroll
    for (int k = 0; k < K3D_STEPS; ++k) v[k] = r0 + k * 32 < m ? __ldcg(yd + r0 + k * 32) : kEmpty;
    uint32_t bits[K3D_STEPS];
    int32_t cw = 0;
#pragma unroll
    for (int k = 0; k < K3D_STEPS; ++k) {
      bits[k] = __ballot_sync(0xffffffffu, v[k] != kEmpty);
      cw += __popc(bits[k]);
    }
    int32_t tot;
    const int32_t run = block_exclusive_sum<K3_THREADS>(lane == 0 ? cw : 0, s_scan, &tot);
    if (tid < 32) {
      const unsigned long long pre = warp_lookback(ws.k3_status, t, (unsigned long long)tot, st);
      if (tid == 0) s_off = pre;
    }
    __syncthreads();
    int64_t pos = (int64_t)s_off + __shfl_sync(0xffffffffu, run, 0);
#pragma unroll
    for (int k = 0; k < K3D_STEPS; ++k) {
      if ((bits[k] >> lane) & 1u) {
        const int64_t r = r0 + k * 32;
        const int64_t pp = pos + __popc(bits[k] & lt);
        if (pp < y_cap) {
          y_idx[pp] = (int32_t)r;
          if (y_val) y_val[pp] = v[k];
        }
        yd[r] = kEmpty;
      }
      pos += __popc(bits[k]);
    }
    if (t == ntiles - 1 && tid == 0) {
      const int64_t total = (int64_t)s_off + tot;
      st->nnz_y = (int32_t)total;
      if (d_nnz_y) *d_nnz_y = (int32_t)total;
      if (total > y_cap) atomicOr(&st->status, ST_CAPACITY);
    }
    __syncthreads();
  }
}

template <int SEM, bool BFS>
__global__ void __launch_bounds__(K3_THREADS, 2)
k3_bucket_merge(Workspace ws, int lwb_lo, int nb_fine, int32_t m, int32_t* y_idx, uint32_t* y_val,
                int32_t y_cap, int32_t* d_nnz_y, uint32_t* mask_update, int only_push,
                int32_t direct_max, int use_cond, cudaGraphConditionalHandle cond,
                int32_t plus_direct_min) {
  pdl_wait();  // the expand step's outputs are complete and visible
  if (only_push && ws.st->dir != 0) return;  // this call runs the pull direction
  if (ws.job) {  // a batched lane: this frontier's outputs
    y_idx = ws.job->y_idx;
    y_val = ws.job->y_val;
    y_cap = ws.job->y_cap;
    d_nnz_y = ws.job->d_nnz_y;
    if (BFS) mask_update = ws.job->visited;
  }
  if (BFS && direct_max > 0 && ws.st->W <= direct_max) {  // K2 ran the level in the direct form
    k3_bfs_direct_close(ws, m, y_idx, d_nnz_y, use_cond, cond);
    return;
  }
  extern __shared__ __align__(16) uint32_t k3_smem[];
  if (SEM == kPlusTimes && !BFS && plus_direct_min > 0 && ws.st->W >= plus_direct_min) {
    k3_plus_direct(ws, m, y_idx, y_val, y_cap, d_nnz_y);
    return;
  }
  constexpr bool kDenseForm = SEM == kPlusTimes || (SEM == kMinSelect2nd && BFS);
  __shared__ int32_t s_scan[K3_THREADS / 32 + 1];
  __shared__ uint32_t s_tk[2];  // this bucket's ticket and the next one's
  __shared__ unsigned long long s_off;
  __shared__ int32_t s_tot;

  DevState* st = ws.st;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int lwb = st->lwb;
  const int sh = lwb - lwb_lo;
  const int32_t wb = 1 << lwb;
  const uint32_t wmask = (uint32_t)wb - 1u;
  const int nw = wb >> 5;
  const int nb = (int)(((int64_t)m + wb - 1) >> lwb);
  uint32_t* spa = k3_smem;
  uint32_t* occ = k3_smem + wb;
  const uint32_t ident = sr_identity<SEM>();
  const uint32_t empty = spa_empty<SEM>();
  const int wpt = nw > K3_THREADS ? nw / K3_THREADS : 1;
  const bool or_always = wb >= (1 << 15);
  const int rpw = wb / K3_WARPS;  // dense form: rows each warp compacts
  const int32_t lvl = BFS ? (ws.job ? ws.job->lvl : st->level) : 0;
  int32_t* const level = BFS ? (ws.job ? ws.job->level : st->bfs_level) : nullptr;
  int32_t* const parent = BFS ? (ws.job ? ws.job->parent : st->bfs_parent) : nullptr;
  const int nhot = ws.nhot;
  // single-source BFS: this level's frontier bitmap (every word is written,
  // zeros for buckets without rows) for a pull at the next level
  uint32_t* fbn = nullptr;
  const int64_t fb_words = ((int64_t)m + 31) / 32;
  if (BFS && !ws.job && st->bfs_fb) fbn = st->bfs_fb + ((lvl & 1) ? fb_words : 0);
  if (BFS && ws.job && ws.job->fb) fbn = ws.job->fb + ((lvl & 1) ? fb_words : 0);

  if (blockIdx.x == 0 && tid == 0) {
    // clear K1's per-call state for the next call
    st->k1_ticket = 0u;
    st->last_maxdeg = st->maxdeg;
    st->last_maskcnt = st->maskcnt;
    st->maxdeg = 0;
    st->maskcnt = 0;
  }
  if (blockIdx.x == 0) {
    const int nt1 = (st->f + K1_TILE - 1) / K1_TILE;
    for (int i = tid; i < nt1; i += K3_THREADS) ws.k1_status[i] = 0ull;
  }

  // tickets hand out the buckets in order; the next one is taken once this
  // one is merged, so that it is in hand by the end of the compaction (every
  // CTA still processes its buckets in ticket order, so the smallest
  // unfinished bucket can always proceed; taking it only after the merge
  // leaves none to CTAs that start late)
  if (tid == 0) s_tk[0] = atomicAdd(&st->k3_ticket, 1u);
  __syncthreads();
  for (int it = 0;; ++it) {
    const uint32_t b = s_tk[it & 1];
    if (b >= (uint32_t)nb) break;
    const int fb0 = (int)(b << sh), fb1 = min((int)(b + 1) << sh, nb_fine);
    const int32_t base = ws.rbase[fb0];
    const int32_t cap = ws.rbase[fb1] - base;
    const int32_t cnt = min(ws.bfill[(size_t)b * BFILL_STRIDE], cap);
    const int hs0 = nhot > 0 ? ws.hot_start[fb0] : 0;
    const int hs1 = nhot > 0 ? ws.hot_start[fb1] : 0;
    const int32_t row0 = (int32_t)(b << lwb);
    int hot_any = 0;
    for (int hs = hs0 + tid; hs < hs1; hs += K3_THREADS) hot_any |= (int)ws.hot_touch[hs];
    const int active = __syncthreads_or(cnt > 0 || hot_any);
    const bool dense = kDenseForm && wb >= K3_DENSE_MIN_WB && (int64_t)cnt * K3_DENSE_DIV >= wb;

    if (active) {
      if (dense) {
        uint4* s4 = reinterpret_cast<uint4*>(spa);
        for (int r = tid; r < (wb >> 2); r += K3_THREADS) s4[r] = make_uint4(empty, empty, empty, empty);
      } else {
        for (int w = tid; w < nw; w += K3_THREADS) occ[w] = 0u;
        if (SEM != kOrAnd) {
          if ((int64_t)cnt * 16 < wb) {
            // partial initialisation: only the SPA slots this bucket touches (Sec. II-F)
            for (int32_t e = tid; e < cnt; e += K3_THREADS) spa[ws.brow[base + e] & wmask] = ident;
            for (int hs = hs0 + tid; hs < hs1; hs += K3_THREADS) spa[ws.hot_rows[hs] - row0] = ident;
          } else {
            for (int r = tid; r < wb; r += K3_THREADS) spa[r] = ident;
          }
        }
      }
      __syncthreads();
      // Step 2 of Algorithm 1: merge the bucket into the SPA.  The bucket's
      // entries [base, base+cnt) are read in aligned 8-entry chunks (one
      // 16-byte load of row ids, two of values), entries outside the range
      // masked off; two chunks per thread are in flight at once.
      {
        constexpr int U = 2;
        const int32_t a0 = base, a1 = base + cnt;
        const int32_t c1 = (a1 + 7) >> 3;
        const uint4* brow4 = reinterpret_cast<const uint4*>(ws.brow);
        const uint4* bval4 = reinterpret_cast<const uint4*>(ws.bval);
        for (int32_t c = (a0 >> 3) + tid; c < c1; c += K3_THREADS * U) {
          uint4 rv[U], va[U], vb[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int32_t cc = c + u * K3_THREADS;
            rv[u] = make_uint4(0u, 0u, 0u, 0u);
            va[u] = rv[u];
            vb[u] = rv[u];
            if (cc < c1) {
              rv[u] = __ldcs(brow4 + cc);
              if (SEM != kOrAnd) {
                va[u] = __ldcs(bval4 + 2 * cc);
                vb[u] = __ldcs(bval4 + 2 * cc + 1);
              }
            }
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int32_t e0 = (c + u * K3_THREADS) << 3;
            const uint32_t rw[4] = {rv[u].x, rv[u].y, rv[u].z, rv[u].w};
            const uint32_t vw[8] = {va[u].x, va[u].y, va[u].z, va[u].w, vb[u].x, vb[u].y, vb[u].z, vb[u].w};
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int32_t e = e0 + j;
              if (e < a0 || e >= a1) continue;
              const uint32_t rr = ((j & 1) ? (rw[j >> 1] >> 16) : (rw[j >> 1] & 0xffffu)) & wmask;
              if (!dense) {
                const uint32_t bit = 1u << (rr & 31);
                // with one CTA per SM (the 128 KB SPA of 32768-row buckets) the
                // dependent test costs more than the extra shared OR it saves
                if (or_always || !(occ[rr >> 5] & bit)) atomicOr(occ + (rr >> 5), bit);
              }
              spa_apply<SEM>(spa, rr, vw[j]);
            }
          }
        }
      }
      // hub rows of this bucket: their products were combined in K2
      for (int hs = hs0 + tid; hs < hs1; hs += K3_THREADS) {
        if (!ws.hot_touch[hs]) continue;
        const uint32_t rr = (uint32_t)(ws.hot_rows[hs] - row0);
        if (!dense) atomicOr(occ + (rr >> 5), 1u << (rr & 31));
        spa_apply<SEM>(spa, rr, ws.hot_val[hs]);
      }
      __syncthreads();
    }
    if (tid == 0) s_tk[(it + 1) & 1] = atomicAdd(&st->k3_ticket, 1u);
    // unique rows of this bucket (|uind_k|), then the offset of the bucket in y
    int32_t c = 0;
    const int w0 = tid * wpt;
    if (dense) {
      // each warp counts its own run of rows (lane 0 carries the count)
      int32_t cw = 0;
      for (int r = warp * rpw + lane; r < (warp + 1) * rpw; r += 32)
        cw += __popc(__ballot_sync(0xffffffffu, spa[r] != empty));
      c = lane == 0 ? cw : 0;
    } else if (active && w0 < nw) {
      for (int w = w0; w < w0 + wpt; ++w) c += __popc(occ[w]);
    }
    int32_t tot;
    int32_t run = block_exclusive_sum<K3_THREADS>(c, s_scan, &tot);
    if (tid < 32) {
      const unsigned long long pre = warp_lookback(ws.k3_status, b, (unsigned long long)tot, st);
      if (tid == 0) {
        s_off = pre;
        s_tot = tot;
      }
    }
    __syncthreads();
    // Step 3: this bucket's rows, ascending, at its offset in y
    if (dense) {
      int64_t pos = (int64_t)s_off + __shfl_sync(0xffffffffu, run, 0);
      const uint32_t lt = (1u << lane) - 1u;
      for (int r0w = warp * rpw; r0w < (warp + 1) * rpw; r0w += 32) {
        const int r = r0w + lane;
        const uint32_t v = spa[r];
        const bool hit = v != empty;
        const uint32_t bits = __ballot_sync(0xffffffffu, hit);
        if (hit) {
          const int64_t p = pos + __popc(bits & lt);
          const int32_t i = row0 + r;
          if (p < y_cap) {
            y_idx[p] = i;
            if (y_val) y_val[p] = v;
          }
          if (BFS) {
            level[i] = lvl;
            parent[i] = (int32_t)v;
          }
        }
        if (BFS && lane == 0) {
          const int64_t gw = (int64_t)b * nw + (r0w >> 5);
          if (bits) mask_update[gw] |= bits;
          if (fbn && gw < fb_words) fbn[gw] = bits;
        }
        pos += __popc(bits);
      }
    } else {
      if (active && w0 < nw) {
        int64_t pos = (int64_t)s_off + run;
        for (int w = w0; w < w0 + wpt; ++w) {
          uint32_t bits = occ[w];
          if (BFS && bits) mask_update[(int64_t)b * nw + w] |= bits;
          while (bits) {
            const int r = (w << 5) + __ffs(bits) - 1;
            bits &= bits - 1u;
            const int32_t i = row0 + r;
            if (pos < y_cap) {
              y_idx[pos] = i;
              if (SEM != kOrAnd && y_val) y_val[pos] = spa[r];
            }
            if (BFS) {
              level[i] = lvl;
              parent[i] = (int32_t)spa[r];
            }
            ++pos;
          }
        }
      }
      if (BFS && fbn && w0 < nw) {
        for (int w = w0; w < w0 + wpt; ++w) {
          const int64_t gw = (int64_t)b * nw + w;
          if (gw < fb_words) fbn[gw] = active ? occ[w] : 0u;
        }
      }
    }
    if (b == (uint32_t)nb - 1u && tid == 0) {
      const int64_t total = (int64_t)s_off + s_tot;
      st->nnz_y = (int32_t)total;
      if (BFS) st->nvisited += (int32_t)total;
      if (d_nnz_y) *d_nnz_y = (int32_t)total;
      if (total > y_cap) atomicOr(&st->status, ST_CAPACITY);
      // a BFS graph's loop: another level while this one found vertices
      if (BFS && use_cond) cudaGraphSetConditional(cond, (total > 0 && st->level <= m) ? 1u : 0u);
    }
    __syncthreads();
  }
}

cudaError_t launch_k3(int sem, bool bfs, const Matrix& A, const Workspace& ws, int lwb_lo,
                      int nb_fine, int32_t* y_idx, uint32_t* y_val, int32_t y_cap, int32_t* d_nnz_y,
                      uint32_t* mask_update, int grid, size_t smem, cudaStream_t s, int only_push,
                      int32_t direct_max, int use_cond, cudaGraphConditionalHandle cond,
                      int32_t plus_direct_min) {
  if (!ws.ydense || bfs || sem != kPlusTimes) plus_direct_min = 0;
  const bool pdl = pdl_allowed(s);
#define K3_ARGS ws, lwb_lo, nb_fine, A.m, y_idx, y_val, y_cap, d_nnz_y, mask_update, only_push, \
                bfs ? direct_max : 0, bfs ? use_cond : 0, cond, plus_direct_min
  if (bfs) {
    launch_after(k3_bucket_merge<kMinSelect2nd, true>, grid, K3_THREADS, smem, s, pdl, K3_ARGS);
  } else if (sem == kPlusTimes) {
    launch_after(k3_bucket_merge<kPlusTimes, false>, grid, K3_THREADS, smem, s, pdl, K3_ARGS);
  } else if (sem == kMinSelect2nd) {
    launch_after(k3_bucket_merge<kMinSelect2nd, false>, grid, K3_THREADS, smem, s, pdl, K3_ARGS);
  } else {
    launch_after(k3_bucket_merge<kOrAnd, false>, grid, K3_THREADS, smem, s, pdl, K3_ARGS);
  }
#undef K3_ARGS
  return cudaGetLastError();
}

__global__ void k_fill_u32(uint32_t* __restrict__ p, int64_t n, uint32_t value) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = value;
}

cudaError_t launch_fill_u32(uint32_t* p, int64_t n, uint32_t value, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
  k_fill_u32<<<grid, 256, 0, s>>>(p, n, value);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------
// create-time: nonzeros per fine row-range bucket (sizes the bucket regions)
// ------------------------------------------------------------------------
__global__ void k_bucket_sizes(const int32_t* __restrict__ rowidx, int64_t nnz, int32_t m,
                               int lwb_lo, int nb_fine, int32_t* __restrict__ counts,
                               unsigned int* __restrict__ bad) {
  extern __shared__ int32_t h[];
  for (int b = threadIdx.x; b < nb_fine; b += blockDim.x) h[b] = 0;
  __syncthreads();
  unsigned int nbad = 0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = rowidx[p];
    if (r < 0 || r >= m) {
      ++nbad;
      continue;
    }
    atomicAdd(&h[r >> lwb_lo], 1);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb_fine; b += blockDim.x)
    if (h[b]) atomicAdd(&counts[b], h[b]);
  if (nbad) atomicAdd(bad, nbad);
}

__global__ void k_row_degrees(const int32_t* __restrict__ rowidx, int64_t nnz, int32_t m,
                              int32_t* __restrict__ deg) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = rowidx[p];
    if (r >= 0 && r < m) atomicAdd(&deg[r], 1);
  }
}

// Hub rows get the ids m + hub index in the row-id copy K2 reads.
__global__ void k_relabel_hubs(const int32_t* __restrict__ rowidx, int64_t nnz,
                               const int32_t* __restrict__ hub_of_row, int32_t m,
                               int32_t* __restrict__ out) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = rowidx[p];
    const int32_t h = (r >= 0 && r < m) ? hub_of_row[r] : -1;
    out[p] = h >= 0 ? m + h : r;
  }
}

cudaError_t launch_relabel_hubs(const Matrix& A, const int32_t* hub_of_row, int32_t* out,
                                cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (A.nnz > 0) k_relabel_hubs<<<sms * 4, 512, 0, s>>>(A.rowidx, A.nnz, hub_of_row, A.m, out);
  return cudaGetLastError();
}

// Flags a column whose row ids do not strictly ascend: one warp per column,
// lanes compare neighbouring entries 32 apart (coalesced).
__global__ void k_rows_unsorted(const int32_t* __restrict__ colptr, const int32_t* __restrict__ rowidx,
                                int32_t n, int32_t* __restrict__ unsorted) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  bool bad = false;
  for (int64_t j = warp; j < n; j += nwarps) {
    const int32_t p1 = colptr[j + 1];
    for (int32_t p = colptr[j] + 1 + lane; p < p1; p += 32) bad |= rowidx[p] <= rowidx[p - 1];
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(unsorted, 1);
}

cudaError_t launch_rows_unsorted(const Matrix& A, int32_t* unsorted, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_rows_unsorted<<<sms * 8, 256, 0, s>>>(A.colptr, A.rowidx, A.jc ? A.nzc : A.n, unsorted);
  return cudaGetLastError();
}

__global__ void k_max_i32(const int32_t* __restrict__ v, int32_t n, int32_t* __restrict__ out) {
  int32_t mx = 0;
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    mx = max(mx, v[i]);
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

cudaError_t launch_row_degrees(const Matrix& A, int32_t* deg, int32_t* maxdeg, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (A.nnz > 0) k_row_degrees<<<sms * 4, 512, 0, s>>>(A.rowidx, A.nnz, A.m, deg);
  k_max_i32<<<sms, 512, 0, s>>>(deg, A.m, maxdeg);
  return cudaGetLastError();
}

cudaError_t launch_bucket_sizes(const Matrix& A, int lwb_lo, int nb_fine, int32_t* counts,
                                unsigned int* bad, cudaStream_t s) {
  size_t smem = sizeof(int32_t) * (size_t)nb_fine;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_bucket_sizes, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_bucket_sizes<<<sms * 2, 1024, smem, s>>>(A.rowidx, A.nnz, A.m, lwb_lo, nb_fine, counts, bad);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------
// attributes and occupancy
// ------------------------------------------------------------------------
cudaError_t set_kernel_attributes(size_t k2_smem, size_t k3_smem_max) {
  cudaError_t e;
#define SET(fn, bytes)                                                                      \
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(bytes)); \
  if (e != cudaSuccess) return e;
#define SET_K2(S)                                            \
  SET((k2_expand_scatter<S, 0, false>), k2_smem);            \
  SET((k2_expand_scatter<S, K2_IMAX / 2, false>), k2_smem);  \
  SET((k2_expand_scatter<S, K2_IMAX, false>), k2_smem);      \
  SET((k2_expand_scatter<S, 0, true>), k2_smem);             \
  SET((k2_expand_scatter<S, K2_IMAX / 2, true>), k2_smem);   \
  SET((k2_expand_scatter<S, K2_IMAX, true>), k2_smem);
  SET_K2(kPlusTimes)
  SET_K2(kMinSelect2nd)
  SET_K2(kOrAnd)
#undef SET_K2
  SET((k3_bucket_merge<kPlusTimes, false>), k3_smem_max);
  SET((k3_bucket_merge<kMinSelect2nd, false>), k3_smem_max);
  SET((k3_bucket_merge<kOrAnd, false>), k3_smem_max);
  SET((k3_bucket_merge<kMinSelect2nd, true>), k3_smem_max);
#undef SET
  return cudaSuccess;
}

int k3_blocks_per_sm(int sem, size_t smem) {
  int nb = 0;
  if (sem == kPlusTimes)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k3_bucket_merge<kPlusTimes, false>, K3_THREADS, smem);
  else if (sem == kMinSelect2nd)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k3_bucket_merge<kMinSelect2nd, false>, K3_THREADS, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k3_bucket_merge<kOrAnd, false>, K3_THREADS, smem);
  return nb > 0 ? nb : 1;
}

int k2_blocks_per_sm(int sem, size_t smem) {
  int nb = 0;
  if (sem == kPlusTimes)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k2_expand_scatter<kPlusTimes, 0, true>, K2_THREADS, smem);
  else if (sem == kMinSelect2nd)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k2_expand_scatter<kMinSelect2nd, 0, true>, K2_THREADS, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k2_expand_scatter<kOrAnd, 0, true>, K2_THREADS, smem);
  return nb > 0 ? nb : 1;
}

}  // namespace spmspv

namespace spmspv {
// BFS level: x values are the vertex ids themselves (select2nd passes the
// parent id), the count comes from the device, and the level advances.
cudaError_t launch_k1_bfs(const Matrix& A, const Workspace& ws, int nb_fine, const int32_t* x_idx,
                          const int32_t* f_dev, int grid, const Sched* sc, cudaStream_t s,
                          const uint32_t* mask, const SelArgs* sel) {
  SelArgs none{};
  k1_work_scan<<<grid, K1_THREADS, 0, s>>>(x_idx, reinterpret_cast<const uint32_t*>(x_idx), 0,
                                           f_dev, A.colptr, A.jc, A.aux, A.aux_shift,
                                           compaction_capacity(A), A.n, A.nnz, ws, nb_fine, kMinSelect2nd,
                                           sc ? sc->id + 1 : 0, sc ? sc->dir : 0, sc ? sc->q : 0,
                                           sc ? sc->lwb : 0, 1, mask, A.m, sel ? *sel : none);
  return cudaGetLastError();
}
}  // namespace spmspv
