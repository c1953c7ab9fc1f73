// Persistent BFS levels for the adaptive schedules of spmspv_bfs (the
// learned selector, SPMSPV_SCHED_AUTO, and the direction-optimizing rule,
// SPMSPV_SCHED_RULE) on a CSC handle.
//
// A high-diameter graph makes a BFS of hundreds of levels with small
// frontiers; run as the plain per-level kernels (work scan -> expand ->
// merge) each level pays their launches and ramp-up, which is most of its
// time.  This kernel, launched once when the search starts, before the BFS
// graph's loop, with every CTA resident (a cooperative launch), runs
// consecutive levels itself, one grid barrier per level.  Such levels are
// push levels in the direct form (both schedules keep a level of at most
// BFS_DIRECT_MAX products on push):
//   - every CTA loads an equal slice of the frontier x and compacts its
//     non-empty columns with their first products; the level's counts
//     (products, non-empty columns, largest column) come from the level
//     before, summed while its vertices were found;
//   - the CTA applies the masked (min, select2nd) product to its slice: one
//     compare-and-swap on the level decides whether a row is new (first
//     finder), found again in this level or reached before, an unsigned min
//     on the parent follows (the parent array is the SPA: -1 is the largest
//     value), and the first finder appends the vertex to the next frontier
//     (one atomic per warp) and adds its column length to the next counts;
//   - a grid barrier closes the level.
// The first level that is too large or too uneven for the direct form is
// left, with all the levels after it, to the graph's loop of plain kernels
// (where the selector or the rule decides each level), its state exactly as
// at the level's start.  Every wait is bounded; a wait that runs out sets
// SPMSPV_DEV_TIMEOUT and the kernel returns.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "device_util.cuh"
#include "handle.cuh"
#include "selector_dev.cuh"
#include "spmspv_internal.cuh"

namespace spmspv {
namespace {

constexpr int FB_THREADS = 512;
constexpr int FB_WARPS = FB_THREADS / 32;
constexpr int FB_CH = 2048;                    // frontier entries of one CTA's slice (4 per thread)
constexpr int FB_QT = 4096;                    // products per tile (8 per thread)
constexpr int FB_IT = FB_QT / FB_THREADS;
constexpr int32_t FB_COL_MAX = 1 << 15;        // a larger selected column goes to the plain kernels
constexpr int32_t FB_F_MAX = 1 << 18;          // so does a larger frontier

struct FusedArgs {
  const int32_t* colptr;
  const int32_t* rowidx;
  int32_t n;
  int64_t nnz;
  uint32_t* visited;
  int32_t* front0;      // the frontier list the plain kernels read and write
  int32_t* front1;      // the other buffer of a level's next frontier
  uint32_t* fb;         // frontier bitmaps [2][ceil(n/32)] (NULL: no pull level can follow)
  DevState* st;
  int32_t direct_max;
};

// Grid barrier (every CTA resident: cooperative launch).  The arrival count
// only grows during a search (reset when it starts).
__device__ bool fused_barrier(DevState* st, uint32_t epoch, int* s_ok) {
  return grid_barrier(&st->fused_count, epoch, &st->status, s_ok);
}

template <typename T, typename Op>
__device__ __forceinline__ T block_reduce(T v, T* sh, Op op) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T r = sh[0];
  for (int i = 1; i < FB_WARPS; ++i) r = op(r, sh[i]);
  return r;
}

__global__ void __launch_bounds__(FB_THREADS, 2) k_bfs_fused(FusedArgs a) {
  __shared__ int32_t s_c0[FB_CH];        // column start of every non-empty entry of the slice
  __shared__ int32_t s_lo[FB_CH + 1];    // its first product in the slice
  __shared__ uint32_t s_x[FB_CH];        // its vertex id (the value select2nd passes on)
  __shared__ uint32_t s_hb[FB_QT / 32];  // entry starts inside a product tile
  __shared__ long long s_red[FB_WARPS];
  __shared__ long long s_cw[FB_WARPS];   // per-warp counts of the next frontier
  __shared__ int32_t s_cfc[FB_WARPS], s_cmd[FB_WARPS];
  __shared__ unsigned long long s_scan[FB_THREADS / 32 + 1];
  __shared__ int s_ok, s_efirst, s_nq;
  __shared__ int32_t s_S;

  DevState* st = a.st;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int32_t G = (int32_t)gridDim.x, c = (int32_t)blockIdx.x, n = a.n;
  int32_t* level = st->bfs_level;    // this search's outputs (set when it started)
  uint32_t* parent = reinterpret_cast<uint32_t*>(st->bfs_parent);
  for (int i = tid; i < FB_QT / 32; i += FB_THREADS) s_hb[i] = 0u;
  // the search's state at this launch (written by the kernels before it)
  int32_t f = __ldcg(&st->nnz_y), L = __ldcg(&st->level), nvis = __ldcg(&st->nvisited);
  const int32_t L0 = L;
  uint32_t epoch = __ldcg(&st->fused_gen);
  long long seen = __ldcg(&st->edges_seen);  // expanded edges (the rule counts them)
  int cur = 0;          // 0: x in front0, 1: x in front1
  bool have = false;    // counts of the current frontier known (from the level before)
  long long W = 0;
  int32_t fc = 0, md = 0;
  for (;;) {
    const int32_t Ln = L + 1;  // the level this iteration discovers
    // (the slice of every CTA must fit its shared arrays)
    if (f == 0 || Ln > n || f > FB_F_MAX || (f + G - 1) / G > FB_CH) break;
    const int32_t* x = cur ? a.front1 : a.front0;
    int32_t* y = cur ? a.front0 : a.front1;
    // ---- this CTA's slice of x: non-empty entries compacted in order with
    // their first product (a packed scan: products low, entries high) ----
    const int32_t E = (f + G - 1) / G;
    const int32_t e0 = min(f, c * E), e1 = min(f, e0 + E);
    constexpr int PER = FB_CH / FB_THREADS;
    int32_t jv[PER], c0v[PER], dv[PER];
    unsigned long long tsum = 0;
    int32_t mxd = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int32_t k = e0 + tid * PER + i;
      jv[i] = 0;
      c0v[i] = 0;
      dv[i] = 0;
      if (k < e1) {
        jv[i] = x[k];
        c0v[i] = __ldg(a.colptr + jv[i]);
        dv[i] = __ldg(a.colptr + jv[i] + 1) - c0v[i];
      }
      tsum += dv[i] > 0 ? (1ull << 32) + (unsigned long long)dv[i] : 0ull;
      mxd = max(mxd, dv[i]);
    }
    unsigned long long tot;
    unsigned long long run = block_exclusive_sum<FB_THREADS>(tsum, s_scan, &tot);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      if (dv[i] > 0) {
        const int q = (int)(run >> 32);
        s_c0[q] = c0v[i];
        s_lo[q] = (int32_t)(run & 0xffffffffull);
        s_x[q] = (uint32_t)jv[i];
        run += (1ull << 32) + (unsigned long long)dv[i];
      }
    }
    if (tid == 0) {
      s_nq = (int)(tot >> 32);
      s_S = (int32_t)(tot & 0xffffffffull);
      s_lo[s_nq] = s_S;
    }
    __syncthreads();  // the slice's entries and sizes, for every thread
    if (!have) {
      // the first level of this launch: its counts from every slice (into the
      // start slot, which K1 zeroes), and this level's counters start at zero
      const long long mxb = block_reduce((long long)mxd, s_red, [](long long p, long long q) { return p > q ? p : q; });
      if (tid == 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&st->fused_w[3]), (unsigned long long)(tot & 0xffffffffull));
        atomicAdd(&st->fused_fc[3], (int32_t)(tot >> 32));
        atomicMax(&st->fused_md[3], (int32_t)mxb);
        if (c == 0) {
          st->fused_cnt[Ln % 3] = 0;
          st->fused_w[Ln % 3] = 0;
          st->fused_fc[Ln % 3] = 0;
          st->fused_md[Ln % 3] = 0;
        }
      }
      if (!fused_barrier(st, ++epoch, &s_ok)) return;
      W = (long long)__ldcg(reinterpret_cast<const unsigned long long*>(&st->fused_w[3]));
      fc = __ldcg(&st->fused_fc[3]);
      md = __ldcg(&st->fused_md[3]);
      have = true;
    }
    if (W > a.direct_max || md > FB_COL_MAX) break;  // the plain kernels take this level
    seen += W;
    // the counters of the level after next start at zero (last read two levels ago)
    if (c == 0 && tid == 0) {
      st->fused_cnt[(Ln + 1) % 3] = 0;
      st->fused_w[(Ln + 1) % 3] = 0;
      st->fused_fc[(Ln + 1) % 3] = 0;
      st->fused_md[(Ln + 1) % 3] = 0;
    }
    int32_t* cnt = &st->fused_cnt[Ln % 3];
    const int nq = s_nq;
    const int32_t S = s_S;
    // ---- the products of this CTA's slice, in the direct form ----
    long long nsum = 0;
    int32_t nfc = 0, nmd = 0;
    for (int32_t P0 = 0; P0 < S; P0 += FB_QT) {
      const int32_t np = min(FB_QT, S - P0);
      for (int q = tid; q < nq; q += FB_THREADS) {
        const int32_t lo = s_lo[q], off = lo - P0;
        if (off > 0 && off < FB_QT) atomicOr(&s_hb[off >> 5], 1u << (off & 31));
        if (lo <= P0 && s_lo[q + 1] > P0) s_efirst = q;
      }
      __syncthreads();
      // gather: lanes on consecutive products, the entry of a product from
      // the starts bitmap (a popcount)
      const int w0 = warp * FB_IT;
      int ent = 0;
      for (int j = lane; j < w0; j += 32) ent += __popc(s_hb[j]);
      ent = __reduce_add_sync(0xffffffffu, ent) + s_efirst;
      const uint32_t le = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
      uint32_t row[FB_IT], val[FB_IT];
#pragma unroll
      for (int i = 0; i < FB_IT; ++i) {
        const int32_t pl = (w0 + i) * 32 + lane;
        const uint32_t hw = s_hb[w0 + i];
        const int e = ent + __popc(hw & le);
        ent += __popc(hw);
        row[i] = 0xffffffffu;
        val[i] = 0u;
        if (pl < np && e < nq) {  // (e < nq always holds; the test keeps the reads in the arrays)
          const int32_t pos = s_c0[e] + (P0 + pl - s_lo[e]);
          if ((uint64_t)pos < (uint64_t)a.nnz) row[i] = (uint32_t)__ldcs(a.rowidx + pos);
          val[i] = s_x[e];
        }
      }
      // one compare-and-swap per product decides: -1 before (first finder),
      // Ln (found in this level too), or an earlier level (nothing to do);
      // the min on the parent follows for the first two
      int32_t old[FB_IT];
#pragma unroll
      for (int i = 0; i < FB_IT; ++i) old[i] = row[i] < (uint32_t)n ? atomicCAS(level + row[i], -1, Ln) : L;
      uint32_t found = 0u;
#pragma unroll
      for (int i = 0; i < FB_IT; ++i) {
        if (row[i] >= (uint32_t)n || (old[i] != -1 && old[i] != Ln)) continue;
        atomicMin(parent + row[i], val[i]);
        if (old[i] == -1) found |= 1u << i;
      }
      const int32_t cf = __popc(found);
      int32_t incl = cf;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t yv = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += yv;
      }
      // the visited bits and the new vertices' column lengths (the next
      // level's counts) are issued before the frontier slots are reserved,
      // so their latency overlaps the reservation's
      int32_t dnew[FB_IT];
#pragma unroll
      for (int i = 0; i < FB_IT; ++i) {
        dnew[i] = 0;
        if (!((found >> i) & 1u)) continue;
        const uint32_t r = row[i];
        atomicOr(a.visited + (r >> 5), 1u << (r & 31));
        dnew[i] = __ldg(a.colptr + r + 1) - __ldg(a.colptr + r);
      }
      int32_t base = 0;
      if (lane == 31 && incl > 0) base = atomicAdd(cnt, incl);
      base = __shfl_sync(0xffffffffu, base, 31) + incl - cf;
#pragma unroll
      for (int i = 0; i < FB_IT; ++i) {
        if (!((found >> i) & 1u)) continue;
        y[base++] = (int32_t)row[i];
        nsum += dnew[i];
        nfc += dnew[i] > 0;
        nmd = max(nmd, dnew[i]);
      }
      __syncthreads();
      for (int j = tid; j < FB_QT / 32; j += FB_THREADS) s_hb[j] = 0u;
      __syncthreads();
    }
    // the next frontier's counts, reduced over the CTA in one pass: one
    // atomic of each kind per CTA
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nsum += __shfl_xor_sync(0xffffffffu, nsum, o);
      nfc += __shfl_xor_sync(0xffffffffu, nfc, o);
      nmd = max(nmd, __shfl_xor_sync(0xffffffffu, nmd, o));
    }
    if (lane == 0) {
      s_cw[warp] = nsum;
      s_cfc[warp] = nfc;
      s_cmd[warp] = nmd;
    }
    __syncthreads();
    if (tid == 0) {
      long long ws = 0;
      int32_t fs = 0, ms = 0;
      for (int i = 0; i < FB_WARPS; ++i) {
        ws += s_cw[i];
        fs += s_cfc[i];
        ms = max(ms, s_cmd[i]);
      }
      if (ws) atomicAdd(reinterpret_cast<unsigned long long*>(&st->fused_w[Ln % 3]), (unsigned long long)ws);
      if (fs) atomicAdd(&st->fused_fc[Ln % 3], fs);
      if (ms) atomicMax(&st->fused_md[Ln % 3], ms);
    }
    if (!fused_barrier(st, ++epoch, &s_ok)) return;
    // ---- the next level: every CTA reads the same counts ----
    f = __ldcg(cnt);
    W = (long long)__ldcg(reinterpret_cast<const unsigned long long*>(&st->fused_w[Ln % 3]));
    fc = __ldcg(&st->fused_fc[Ln % 3]);
    md = __ldcg(&st->fused_md[Ln % 3]);
    nvis += f;
    L = Ln;
    cur ^= 1;
    if (c == 0 && tid == 0) {
      st->level = L;
      st->nnz_y = f;
      st->nvisited = nvis;
      st->edges_seen = seen;
    }
  }
  // a pull level may follow: it reads the frontier bitmap of the last level
  // this kernel ran (cleared, then set from that level's vertices)
  if (a.fb && L > L0 && f > 0) {
    const int64_t words = ((int64_t)n + 31) / 32;
    uint32_t* fbx = a.fb + ((L & 1) ? words : 0);
    for (int64_t w = (int64_t)c * FB_THREADS + tid; w < words; w += (int64_t)G * FB_THREADS) fbx[w] = 0u;
    if (!fused_barrier(st, ++epoch, &s_ok)) return;
    const int32_t* xl = cur ? a.front1 : a.front0;
    for (int32_t k = c * FB_THREADS + tid; k < f; k += G * FB_THREADS) {
      const int32_t v = xl[k];
      atomicOr(fbx + (v >> 5), 1u << (v & 31));
    }
  }
  if (c == 0 && tid == 0) st->fused_gen = epoch;
  // the plain kernels read the frontier from front0
  if (cur)
    for (int32_t k = c * FB_THREADS + tid; k < f; k += G * FB_THREADS) a.front0[k] = a.front1[k];
}

}  // namespace

int fused_bfs_grid(const spmspv_handle* h) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bfs_fused, FB_THREADS, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return std::min(nb, 2) * h->sm_count;
}

// One launch per learned search, before its graph (cooperative: every CTA
// resident, which the grid barrier needs).
cudaError_t launch_bfs_fused(const spmspv_handle* h, int grid, cudaStream_t s) {
  FusedArgs a;
  a.colptr = h->A.colptr;
  a.rowidx = h->A.rowidx;
  a.n = h->A.n;
  a.nnz = h->A.nnz;
  a.visited = h->bfs_visited;
  a.front0 = h->bfs_front;
  a.front1 = h->bfs_front2;
  a.fb = pull_available(h, kMinSelect2nd) ? h->bfs_fb : nullptr;
  a.st = h->ws.st;
  a.direct_max = BFS_DIRECT_MAX;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(FB_THREADS);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_bfs_fused, a);
}

}  // namespace spmspv
