// Pull direction: the matrix-driven form of SpMSpV (Sec. II-B), used as the
// alternative to the bucketed push form when x is dense enough.
//
//   P1 k_pull_scatter  x (list) -> frontier bitmap xbits + dense values xdense
//   P2 k_pull_rows     for every row i allowed by the mask, y(i) = (+) over the
//                      row's entries A(i,j) with x(j) present of A(i,j) (x) x(j);
//                      rows are read from the CSC as CSR, so A must be pattern-
//                      symmetric (values symmetric too for (+,*)); y is written
//                      in row order (block scan + decoupled look-back over tiles)
//   P3 k_pull_clear    clears xbits for the next call
//
// One thread owns one 32-row word of the output (and of the mask), so the
// mask and BFS visited updates need no atomics.  With row ids ascending in
// every column and x(j) = j (BFS frontiers), the first frontier neighbour is
// the minimum, so (min, select2nd) stops there; (or, and) stops at any.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "device_util.cuh"
#include "handle.cuh"
#include "spmspv_internal.cuh"

namespace spmspv {

namespace {

__device__ __forceinline__ bool active_dir(const DevState* st, int only_pull) {
  return !only_pull || st->dir == 1;
}

// x -> bitmap + dense values.  Also resets the pull kernel's ticket and
// look-back words for this call.
__global__ void k_pull_scatter(const int32_t* __restrict__ x_idx, const uint32_t* __restrict__ x_val,
                               int f_host, const int32_t* __restrict__ f_dev, int32_t n,
                               uint32_t* __restrict__ xbits, uint32_t* __restrict__ xdense,
                               unsigned long long* __restrict__ pull_status, int ntiles,
                               DevState* st, int only_pull) {
  if (!active_dir(st, only_pull)) return;
  const int f = f_dev ? *f_dev : f_host;
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < ntiles; i += blockDim.x) pull_status[i] = 0ull;
    if (threadIdx.x == 0) st->pull_ticket = 0u;
  }
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < f; k += gridDim.x * blockDim.x) {
    const int32_t j = x_idx[k];
    if (j < 0 || j >= n) {
      atomicOr(&st->status, ST_INDEX);
      continue;
    }
    atomicOr(xbits + (j >> 5), 1u << (j & 31));
    xdense[j] = x_val ? x_val[k] : (uint32_t)j;
  }
}

__global__ void k_pull_clear(uint32_t* __restrict__ xbits, int32_t words, const DevState* st,
                             int only_pull) {
  if (!active_dir(st, only_pull)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < words; i += gridDim.x * blockDim.x)
    xbits[i] = 0u;
}

template <int SEM, bool BFS>
__global__ void __launch_bounds__(PULL_THREADS)
k_pull_rows(const int32_t* __restrict__ colptr, const int32_t* __restrict__ rowidx,
            const float* __restrict__ val, int32_t m, const uint32_t* __restrict__ xbits,
            const uint32_t* __restrict__ xdense, const uint32_t* mask, int mask_comp,
            int early_exit, int32_t* __restrict__ y_idx, uint32_t* __restrict__ y_val,
            int32_t y_cap, int32_t* __restrict__ d_nnz_y, uint32_t* visited,  // a BFS passes one
                                                                            // bitmap as mask and visited
            Workspace ws, int ntiles, int only_pull, int use_cond, cudaGraphConditionalHandle cond) {
  __shared__ uint32_t s_val[PULL_THREADS * 33];
  __shared__ int32_t s_scan[PULL_THREADS / 32 + 1];
  __shared__ uint32_t s_tile;
  __shared__ unsigned long long s_off;
  __shared__ int32_t s_tot;
  DevState* st = ws.st;
  if (!active_dir(st, only_pull)) return;
  const int tid = threadIdx.x;
  const Job* job = ws.job;  // a batched lane's BFS level (only BFS jobs come here)
  int32_t lvl = BFS ? (job ? job->lvl : st->level) : 0;
  int32_t* level = BFS ? (job ? job->level : st->bfs_level) : nullptr;
  int32_t* parent = BFS ? (job ? job->parent : st->bfs_parent) : nullptr;
  uint32_t* fbase = BFS ? (job ? job->fb : st->bfs_fb) : nullptr;
  if (BFS && job) {
    visited = job->visited;
    mask = job->visited;
    mask_comp = 1;
    y_idx = job->y_idx;
    y_val = nullptr;
    y_cap = job->y_cap;
    d_nnz_y = job->d_nnz_y;
  }
  // BFS: x is the previous level's frontier bitmap, x(j) = j; this level's
  // discoveries go to the other bitmap (every word is written)
  uint32_t* fb_next = nullptr;
  if (BFS && fbase) {
    const size_t words = ((size_t)m + 31) / 32;
    xbits = fbase + (((lvl - 1) & 1) ? words : 0);
    fb_next = fbase + ((lvl & 1) ? words : 0);
  }
  if (blockIdx.x == 0) {
    // this kernel ends the call: clear the work scan's per-call state
    if (tid == 0) {
      st->k1_ticket = 0u;
      st->last_maxdeg = st->maxdeg;
      st->last_maskcnt = st->maskcnt;
      st->maxdeg = 0;
      st->maskcnt = 0;
    }
    const int nt1 = (st->f + K1_TILE - 1) / K1_TILE;
    for (int i = tid; i < nt1; i += PULL_THREADS) ws.k1_status[i] = 0ull;
  }
  if (BFS && (!fbase || (job && job->b < 0))) return;  // an empty lane job: nothing to find
  const uint32_t ident = SEM == kMinSelect2nd ? 0x7fffffffu : 0u;
  for (;;) {
    if (tid == 0) s_tile = atomicAdd(&st->pull_ticket, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= (uint32_t)ntiles) break;
    const int32_t w = (int32_t)tile * PULL_THREADS + tid;  // this thread's 32-row word
    const int32_t r0 = w * 32;
    uint32_t found = 0u;
    if (r0 < m) {
      uint32_t allowed = 0xffffffffu;
      if (mask) allowed = mask_comp ? ~mask[w] : mask[w];
      if (m - r0 < 32) allowed &= (1u << (m - r0)) - 1u;
      while (allowed) {
        const int b = __ffs(allowed) - 1;
        allowed &= allowed - 1u;
        const int32_t r = r0 + b;
        const int32_t p1 = colptr[r + 1];
        uint32_t acc = ident;
        bool hit = false;
        for (int32_t p = colptr[r]; p < p1; ++p) {
          const int32_t j = rowidx[p];
          if (!((xbits[j >> 5] >> (j & 31)) & 1u)) continue;
          hit = true;
          if (SEM == kOrAnd) break;
          const uint32_t xv = BFS ? (uint32_t)j : xdense[j];
          if (SEM == kMinSelect2nd) {
            if ((int)xv < (int)acc) acc = xv;
            if (early_exit) break;
          } else {
            const float a = val ? val[p] : 1.0f;
            acc = __float_as_uint(__uint_as_float(acc) + __fmul_rn(a, __uint_as_float(xv)));
          }
        }
        if (hit) {
          found |= 1u << b;
          s_val[tid * 33 + b] = acc;
        }
      }
    }
    // ordered compaction: this tile's rows at its offset in y
    int32_t tot;
    const int32_t c = __popc(found);
    int32_t run = 0;
    {
      // block exclusive scan of c
      const int lane = tid & 31, wid = tid >> 5;
      int32_t x = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) s_scan[wid] = x;
      __syncthreads();
      if (wid == 0) {
        const int32_t v = lane < PULL_THREADS / 32 ? s_scan[lane] : 0;
        int32_t vi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int32_t y = __shfl_up_sync(0xffffffffu, vi, o);
          if (lane >= o) vi += y;
        }
        if (lane < PULL_THREADS / 32) s_scan[lane] = vi - v;
        if (lane == PULL_THREADS / 32 - 1) s_scan[PULL_THREADS / 32] = vi;
      }
      __syncthreads();
      run = s_scan[wid] + x - c;
      tot = s_scan[PULL_THREADS / 32];
    }
    if (tid < 32) {
      const unsigned long long pre = warp_lookback(ws.pull_status, tile, (unsigned long long)tot, st);
      if (tid == 0) {
        s_off = pre;
        s_tot = tot;
      }
    }
    __syncthreads();
    int64_t pos = (int64_t)s_off + run;
    if (BFS && found) visited[w] |= found;
    if (BFS && r0 < m) fb_next[w] = found;
    for (uint32_t bits = found; bits; bits &= bits - 1u) {
      const int b = __ffs(bits) - 1;
      const int32_t i = r0 + b;
      const uint32_t v = s_val[tid * 33 + b];
      if (pos < y_cap) {
        y_idx[pos] = i;
        if (SEM != kOrAnd && y_val) y_val[pos] = v;
      }
      if (BFS) {
        level[i] = lvl;
        parent[i] = (int32_t)v;
      }
      ++pos;
    }
    if (tile == (uint32_t)ntiles - 1u && tid == 0) {
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

}  // namespace

int pull_available(const spmspv_handle* h, int sem) {
  if (!h->xbits || h->A.m != h->A.n) return 0;
  if (sem == kPlusTimes) return (h->flags & SPMSPV_CSC_SYMMETRIC) == SPMSPV_CSC_SYMMETRIC;
  return (h->flags & SPMSPV_CSC_PATTERN_SYMMETRIC) != 0;
}

cudaError_t launch_pull(const spmspv_handle* h, int sem, bool bfs, const int32_t* x_idx,
                        const uint32_t* x_val, int f, const int32_t* f_dev, const uint32_t* mask,
                        int mask_comp, int early_exit, int32_t* y_idx, uint32_t* y_val,
                        int32_t y_cap, int32_t* d_nnz_y, uint32_t* visited, int only_pull,
                        cudaStream_t s) {
  const int32_t n = h->A.n, m = h->A.m;
  const int words = (n + 31) / 32;
  const int sgrid = f_dev ? h->sm_count * 4
                          : std::max(1, std::min(h->sm_count * 4, (f + 255) / 256));
  k_pull_scatter<<<sgrid, 256, 0, s>>>(x_idx, x_val, f, f_dev, n, h->xbits, h->xdense,
                                       h->pull_status, h->pull_tiles, h->ws.st, only_pull);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, std::min(h->pull_tiles, h->sm_count * 8));
#define PULL_ARGS h->A.colptr, h->A.rowidx, h->A.val, m, h->xbits, h->xdense, mask, mask_comp, \
                  early_exit, y_idx, y_val, y_cap, d_nnz_y, visited, h->ws, h->pull_tiles, only_pull, 0, 0
  if (bfs) k_pull_rows<kMinSelect2nd, true><<<grid, PULL_THREADS, 0, s>>>(PULL_ARGS);
  else if (sem == kPlusTimes) k_pull_rows<kPlusTimes, false><<<grid, PULL_THREADS, 0, s>>>(PULL_ARGS);
  else if (sem == kMinSelect2nd) k_pull_rows<kMinSelect2nd, false><<<grid, PULL_THREADS, 0, s>>>(PULL_ARGS);
  else k_pull_rows<kOrAnd, false><<<grid, PULL_THREADS, 0, s>>>(PULL_ARGS);
#undef PULL_ARGS
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_pull_clear<<<std::max(1, std::min(h->sm_count * 4, (words + 255) / 256)), 256, 0, s>>>(
      h->xbits, words, h->ws.st, only_pull);
  return cudaGetLastError();
}

// BFS level in the pull direction: the frontier is the previous level's
// bitmap (written by K3 or by this kernel), so only the row kernel runs; the
// work scan of the level has reset the pull look-back state.
cudaError_t launch_pull_rows_bfs(const spmspv_handle* h, int early_exit, int only_pull, cudaStream_t s,
                                 cudaGraphConditionalHandle cond) {
  // a persistent grid: the tiles are handed out by a ticket, and when the
  // learned schedule picks push the kernel's CTAs only start and return
  const int grid = std::max(1, std::min(h->pull_tiles, h->sm_count * (only_pull ? 2 : 8)));
  k_pull_rows<kMinSelect2nd, true><<<grid, PULL_THREADS, 0, s>>>(
      h->A.colptr, h->A.rowidx, h->A.val, h->A.m, nullptr, nullptr, h->bfs_visited, 1, early_exit,
      h->bfs_front, nullptr, h->A.n, &h->ws.st->nnz_y, h->bfs_visited, h->ws, h->pull_tiles, only_pull,
      1, cond);
  return cudaGetLastError();
}

cudaError_t launch_pull_rows_lane(const spmspv_handle* sub, int early_exit, cudaStream_t s) {
  // the lanes share the GPU: fewer CTAs per lane than a lone call takes
  const int grid = std::max(1, std::min(sub->pull_tiles, sub->sm_count * 2));
  k_pull_rows<kMinSelect2nd, true><<<grid, PULL_THREADS, 0, s>>>(
      sub->A.colptr, sub->A.rowidx, sub->A.val, sub->A.m, nullptr, nullptr, nullptr, 1, early_exit,
      nullptr, nullptr, 0, nullptr, nullptr, sub->ws, sub->pull_tiles, 1, 0, 0);
  return cudaGetLastError();
}

int run_pull_if_available(spmspv_handle* h, int sem, const int32_t* x_idx, const uint32_t* x_val,
                          int f, const uint32_t* mask, int mask_comp, const Sched& sc,
                          int32_t* y_idx, uint32_t* y_val, int32_t y_cap, int32_t* d_nnz_y,
                          cudaStream_t s, int early_exit) {
  (void)sc;
  if (!pull_available(h, sem)) return -1;
  prof_call_begin(h, s);
  cudaError_t e = launch_pull(h, sem, false, x_idx, x_val, f, nullptr, mask, mask_comp, early_exit, y_idx,
                              y_val, y_cap, d_nnz_y, nullptr, 0, s);
  if (e != cudaSuccess) return cuda_fail(e, "pull launch");
  prof_mark(h, SPMSPV_STAGE_PULL, s);
  return SPMSPV_OK;
}

cudaError_t alloc_pull_buffers(spmspv_handle* h) {
  const int32_t n = h->A.n;
  h->pull_tiles = (int)(((int64_t)h->A.m + PULL_ROWS - 1) / PULL_ROWS);
  cudaError_t e = cudaMalloc(&h->xbits, sizeof(uint32_t) * (((size_t)n + 31) / 32));
  if (e == cudaSuccess) e = cudaMalloc(&h->xdense, sizeof(uint32_t) * (size_t)n);
  if (e == cudaSuccess) e = cudaMalloc(&h->pull_status, sizeof(unsigned long long) * (size_t)h->pull_tiles);
  if (e == cudaSuccess) e = cudaMemset(h->xbits, 0, sizeof(uint32_t) * (((size_t)n + 31) / 32));
  if (e == cudaSuccess) {
    h->ws.pull_status = h->pull_status;
    h->ws.pull_tiles = h->pull_tiles;
  }
  return e;
}

void release_extras(spmspv_handle* h) {
  cudaFree(h->xbits);
  cudaFree(h->xdense);
  cudaFree(h->pull_status);
  cudaFree(h->bfs_front);
  cudaFree(h->bfs_front2);
  cudaFree(h->bfs_slice);
  cudaFree(h->bfs_visited);
  cudaFree(h->bfs_fb);
  cudaFree(h->bfs_count);
  h->xbits = nullptr;
  h->xdense = nullptr;
  h->pull_status = nullptr;
  h->bfs_front = nullptr;
  h->bfs_front2 = nullptr;
  h->bfs_slice = nullptr;
  h->fused_grid = 0;
  h->bfs_visited = nullptr;
  h->bfs_fb = nullptr;
  h->bfs_count = nullptr;
}

}  // namespace spmspv
