// Batched SpMSpV as one persistent launch: B independent products
// y_b <- A (+).(x) x_b [under mask_b], every frontier's work in one shared
// pool of thread blocks.
//
// The paper runs one product per call and notes that small calls are mostly
// overhead (Sec. I, Sec. III-A).  Here the batch is one cooperative kernel
// whose CTAs are all resident and pass through phases separated by grid
// barriers (bounded waits), taking work items from device tickets:
//
//   1 scan      x entries in chunks of K6_CH per frontier: the column lengths
//               (Algorithm 2's role), a prefix sum per frontier (decoupled
//               look-back along the frontier's chunks), compaction of the
//               entries with a non-empty column, W_b = the frontier's products.
//   2 plan      one CTA classifies the frontiers: W_b = 0 (empty y), small
//               (W_b <= QMAX products: one CTA does the whole product) and
//               large (tiles of q products, buckets); it numbers the tiles of
//               the large frontiers and splits them into waves whose bucket
//               entries fit the storage.
//   3 tiles     the first x entry of every tile (a merge-path split within
//               each large frontier).
//   per wave:
//   4 expand    Step 1 of Algorithm 1 for every tile of the wave (gather,
//               multiply, mask, count per row-range bucket, stage by bucket in
//               shared memory, write the tile's products in bucket order to
//               the tile's own slot of the storage, with the tile's bucket
//               offsets); before the first wave's tiles, every small frontier
//               is done by one CTA: its products are sorted by row in shared
//               memory (bitonic network), equal rows combined with the
//               semiring's add, and y_b written.
//   5 merge     Steps 2 and 3 for every (frontier, bucket) of the wave: the
//               bucket's runs in all tiles of its frontier are merged into a
//               shared-memory SPA, and its rows written in ascending order at
//               the offset given by a look-back along the frontier's buckets
//               (tasks handed out bucket-major, so that a bucket's
//               predecessor in its chain started one round earlier).
//
// Bucket keys are (frontier, row block): the buckets of different frontiers
// never mix, and a frontier's bucket runs sit in the slots of its own tiles,
// so no bucket capacity has to be reserved and no global atomic places a run.
// Hub rows (the handle's relabelled row ids) are summed per tile in shared
// memory and staged once per tile, so a merge task sees a hub row at most
// once per tile of its frontier.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "device_util.cuh"
#include "expand_dev.cuh"
#include "handle.cuh"
#include "spmspv_internal.cuh"

namespace spmspv {
namespace {

constexpr int K6_THREADS = 512;
constexpr int K6_WARPS = K6_THREADS / 32;
constexpr int K6_CI = 4;                              // x entries per thread in a scan chunk
constexpr int K6_CH = K6_THREADS * K6_CI;             // x entries per scan chunk
constexpr int K6_SMALL_MAX = QMAX;                    // products of a frontier one CTA sorts
constexpr int K6_SEGMAX = 2048;                       // tile runs a merge task lists at once
constexpr int K6_DENSE_DIV = 8;                       // dense SPA when entries >= rows / 8
constexpr int K6_DENSE_MIN_WB = 32 * K6_WARPS;        // every warp compacts whole 32-row words
constexpr int K6_NB_MAX = 2048;                       // buckets per frontier
constexpr int K6_STAMPS = 32;                         // phase clock stamps kept per launch

__host__ __device__ constexpr int k6_pad(int e) { return e + (e >> 5); }

// Counters of one launch (zeroed before it) and what the plan found.
struct K6State {
  uint32_t bar;        // grid barrier arrivals
  uint32_t tk_scan;    // scan chunk tickets
  int32_t n_small;
  int32_t n_large;
  int32_t n_tiles;     // tiles of the large (bucketed) frontiers; the direct ones' follow
  int32_t n_waves;
  int32_t n_direct;    // frontiers in the direct form
  int32_t n_dwaves;    // their waves (at most dslots frontiers each)
  long long padded;    // products of the large frontiers with their tiles rounded up
  unsigned long long t[K6_STAMPS];  // device clock (ns): CTA 0 at its start, after each grid
                                    // barrier (slot = the barrier's number) and at its end (last slot)
};

struct K6Args {
  // batch (device arrays of the caller)
  int32_t B;
  const int32_t* x_off;
  const int32_t* x_idx;
  const uint32_t* x_val;
  const uint32_t* masks;  // complemented masks, frontier b's at masks + b*mask_stride
  int64_t mask_stride;
  int x_ids;              // (min, select2nd): every x value is below INT32_MAX (vertex ids)
  const int32_t* y_off;
  const int32_t* y_cap;
  int32_t* y_idx;
  uint32_t* y_val;
  int32_t* d_nnz_y;
  // matrix
  const int32_t* colptr;
  const int32_t* rowidx;    // row ids as stored (the one-CTA small frontiers)
  const int32_t* rowidx_t;  // row ids of the tiles: hub rows relabelled to m + hub index
  int nhot;                 // hub rows (0: none; rowidx_t == rowidx)
  const int32_t* hot_rows;  // [nhot] their row ids
  const float* val;
  const int32_t* jc;
  const int32_t* aux;
  int aux_shift;
  int32_t m, n;
  int64_t nnz;
  // schedule
  int lwb;        // log2 bucket rows
  int nb;         // buckets per frontier
  int q;          // products per tile of a large frontier
  int64_t win;    // wave window: a wave takes the large frontiers whose padded start lies in it
  int32_t nc;     // scan chunks
  int32_t tw;     // row stride of the tile offset table (tile slots of one wave)
  int32_t nw_cap;
  int32_t tiles_cap;
  // direct form of the frontiers with at least direct_min products ((+,*);
  // (min, select2nd) with x_ids)
  int32_t direct_min;       // 0: no direct form
  int32_t dslots;           // accumulators: frontiers of one direct wave
  uint32_t* dacc;           // [dslots][m] dense accumulators, the empty mark in every row between launches
  unsigned long long* dstat;  // [dslots][nrt] look-back words of the compaction
  int32_t nrt;              // compaction row tiles per accumulator
  int32_t* ld;              // [B] direct frontier ids in order
  int32_t* fdi;             // [B] direct index of each direct frontier
  int32_t* dwt0;            // [B + 2] first tile of each direct wave
  int32_t dw_cap;
  // work arrays
  K6State* st;
  uint32_t* tk;             // [2 * (nw_cap + dw_cap)] expand and merge tickets per wave
  int32_t* wt0;             // [nw_cap + 1] first tile of each wave
  int32_t* wl0;             // [nw_cap + 1] first large frontier of each wave
  unsigned long long* cstat;  // [nc] scan look-back words
  const int32_t* xp;        // [B+1] x entries before frontier b
  const int32_t* cp;        // [B+1] scan chunks before frontier b
  int32_t* fW;              // [B] products of frontier b
  int32_t* ffc;             // [B] its x entries with a non-empty column
  int32_t* ftb;             // [B] its first tile (large frontiers)
  int32_t* lb;              // [B] large frontier ids in order
  int32_t* sl;              // [B] small frontier ids
  int32_t* cw;              // [F] product offset of each compacted entry in its frontier
  int32_t* cb;              // [F] first position of its column
  uint32_t* cx;             // [F] its x value
  int32_t* tk0;             // [tiles_cap] compacted entry holding a tile's first product
  int32_t* tf;              // [tiles_cap] frontier of each tile
  uint16_t* brow;           // [capw] bucket entries of one wave: row inside the bucket
  uint32_t* bval;           // [capw] their values
  int32_t* toff;            // [(nb+1) * tw] tile slot s, bucket r: run start toff[r*tw + s]
  unsigned long long* bstat;  // [B * nb] merge look-back words (per large frontier, per bucket)
  uint32_t* status;         // the handle's sticky status word
};

// Shared memory of the phases (one dynamic buffer, laid out per phase).
__host__ __device__ constexpr size_t k6_smem_scan() { return 3 * sizeof(int32_t) * (size_t)k6_pad(K6_CH); }
__host__ __device__ constexpr size_t k6_smem_expand(int nb) {
  return sizeof(int32_t) * (QMAX + 1) + sizeof(uint32_t) * (QMAX + 1) + sizeof(uint32_t) * (QMAX / 32) +
         sizeof(int32_t) * ((size_t)nb + 1) + sizeof(uint32_t) * HOT_MAX * 2 + sizeof(uint32_t) * (HOT_MAX / 32);
}
__host__ __device__ constexpr size_t k6_smem_merge(int lwb) {
  return ((size_t)1 << lwb) * sizeof(uint32_t) + (((size_t)1 << lwb) / 32) * sizeof(uint32_t) +
         ((size_t)K6_SEGMAX * 3 + 1) * sizeof(int32_t);
}
size_t k6_smem(int lwb, int nb) {
  return std::max(k6_smem_scan(), std::max(k6_smem_expand(nb), k6_smem_merge(lwb)));
}

struct K6Shared {
  unsigned long long scan[K6_WARPS + 1];
  int32_t iscan[K6_WARPS + 1];
  unsigned long long prefix;
  uint32_t item;
  int32_t b;
  int32_t kept;
  int32_t tot;
  long long off;
  int ok;
};

__device__ __forceinline__ unsigned long long k6_clock() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier number `epoch`; CTA 0 stamps the time it passed it.
__device__ __forceinline__ bool k6_barrier(const K6Args& a, uint32_t epoch, K6Shared& sh) {
  const bool ok = grid_barrier(&a.st->bar, epoch, a.status, &sh.ok);
  if (blockIdx.x == 0 && threadIdx.x == 0 && epoch < K6_STAMPS - 1) a.st->t[epoch] = k6_clock();
  return ok;
}

// ---------------------------------------------------------------------------
// phase 1: per-frontier work scan
// ---------------------------------------------------------------------------
constexpr unsigned long long K6_CNT_ONE = 1ull << 31;
constexpr unsigned long long K6_SUM_MASK = (1ull << 31) - 1;

// the frontier of scan chunk c: the largest b < B with cp[b] <= c
__device__ __forceinline__ int32_t k6_frontier_of_chunk(const int32_t* cp, int32_t B, int32_t c) {
  int32_t lo = 0, hi = B - 1;
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (__ldg(cp + mid) <= c) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ void k6_scan(const K6Args& a, unsigned char* smem, K6Shared& sh) {
  int32_t* s_deg = (int32_t*)smem;
  int32_t* s_c0 = s_deg + k6_pad(K6_CH);
  uint32_t* s_xv = (uint32_t*)(s_c0 + k6_pad(K6_CH));
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) {
      const uint32_t c = atomicAdd(&a.st->tk_scan, 1u);
      sh.item = c;
      sh.b = c < (uint32_t)a.nc ? k6_frontier_of_chunk(a.cp, a.B, (int32_t)c) : -1;
    }
    __syncthreads();
    const uint32_t c = sh.item;
    if (c >= (uint32_t)a.nc) break;
    const int32_t b = sh.b;
    const int32_t lc = (int32_t)c - a.cp[b];
    const int32_t xb = a.xp[b];
    const int32_t cnt = a.xp[b + 1] - xb;
    const int32_t i0 = lc * K6_CH;
    const int32_t ne = min(K6_CH, cnt - i0);
    const int64_t xo = (int64_t)a.x_off[b] + i0;
    // striped, coalesced loads of x, then the column ranges
    int32_t jj[K6_CI];
    uint32_t xv[K6_CI];
#pragma unroll
    for (int i = 0; i < K6_CI; ++i) {
      const int e = i * K6_THREADS + tid;
      jj[i] = -1;
      xv[i] = 0u;
      if (e < ne) {
        jj[i] = a.x_idx[xo + e];
        xv[i] = a.x_val ? a.x_val[xo + e] : (uint32_t)jj[i];
      }
    }
#pragma unroll
    for (int i = 0; i < K6_CI; ++i) {
      const int e = i * K6_THREADS + tid;
      int32_t c0 = 0, c1 = 0;
      if (e < ne) {
        if (jj[i] >= 0 && jj[i] < a.n) col_range(a.colptr, a.jc, a.aux, a.aux_shift, jj[i], c0, c1);
        else atomicOr(a.status, ST_INDEX);
      }
      s_deg[k6_pad(e)] = c1 - c0;
      s_c0[k6_pad(e)] = c0;
      s_xv[k6_pad(e)] = xv[i];
    }
    __syncthreads();
    // blocked: thread owns entries [tid*CI, tid*CI + CI)
    unsigned long long tsum = 0;
#pragma unroll
    for (int i = 0; i < K6_CI; ++i) {
      const int d = s_deg[k6_pad(tid * K6_CI + i)];
      tsum += (d > 0 ? K6_CNT_ONE : 0ull) + (unsigned long long)d;
    }
    unsigned long long btot;
    const unsigned long long texcl = block_exclusive_sum<K6_THREADS>(tsum, sh.scan, &btot);
    if (tid < 32) {
      const unsigned long long pre = warp_lookback(a.cstat + a.cp[b], (uint32_t)lc, btot, a.status);
      if (tid == 0) sh.prefix = pre;
    }
    __syncthreads();
    unsigned long long run = sh.prefix + texcl;
#pragma unroll
    for (int i = 0; i < K6_CI; ++i) {
      const int e = tid * K6_CI + i;
      const int d = s_deg[k6_pad(e)];
      if (d > 0) {
        const int32_t qk = (int32_t)((run >> 31) & K6_SUM_MASK);
        const int32_t w = (int32_t)(run & K6_SUM_MASK);
        if (qk < cnt && (int64_t)w + d <= a.nnz) {
          a.cw[xb + qk] = w;
          a.cb[xb + qk] = s_c0[k6_pad(e)];
          a.cx[xb + qk] = s_xv[k6_pad(e)];
        } else {
          atomicOr(a.status, ST_INDEX);  // more products than nonzeros: repeated x indices
        }
        run += K6_CNT_ONE + (unsigned long long)d;
      }
    }
    if (i0 + ne == cnt && tid == 0) {  // the frontier's last chunk: its totals
      const unsigned long long tot = sh.prefix + btot;
      int32_t fc = (int32_t)((tot >> 31) & K6_SUM_MASK);
      int32_t W = (int32_t)(tot & K6_SUM_MASK);
      if (fc > cnt || (int64_t)W > a.nnz) {
        atomicOr(a.status, ST_INDEX);
        fc = 0;
        W = 0;
      }
      a.fW[b] = W;
      a.ffc[b] = fc;
    }
    __syncthreads();
  }
}


// ---------------------------------------------------------------------------
// phase 2: the plan (one CTA)
// ---------------------------------------------------------------------------
// Packed per-frontier counts: tiles in bits [0,32), large in [32,48), small in [48,64).
__device__ void k6_plan(const K6Args& a, K6Shared& sh) {
  const int tid = threadIdx.x;
  int64_t tiles = 0;
  int32_t nlarge = 0, nsmall = 0;
  for (int32_t base = 0; base < a.B; base += K6_THREADS) {
    const int32_t b = base + tid;
    int32_t W = 0;
    if (b < a.B) {
      if (a.cp[b] < a.cp[b + 1]) {
        W = __ldcg(a.fW + b);
      } else {  // no x entries: no chunk wrote the totals
        a.fW[b] = 0;
        a.ffc[b] = 0;
      }
    }
    const bool direct = a.direct_min > 0 && W > K6_SMALL_MAX && W >= a.direct_min;
    const bool large = W > K6_SMALL_MAX && !direct;
    const bool small = W > 0 && W <= K6_SMALL_MAX;
    const unsigned long long T = large ? (unsigned long long)(((int64_t)W + a.q - 1) / a.q) : 0ull;
    const unsigned long long v = T | ((unsigned long long)(large ? 1 : 0) << 32) |
                                 ((unsigned long long)(small ? 1 : 0) << 48);
    unsigned long long tot;
    const unsigned long long ex = block_exclusive_sum<K6_THREADS>(v, sh.scan, &tot);
    if (b < a.B) {
      if (large) {
        const int64_t tb = tiles + (int64_t)(ex & 0xffffffffull);
        a.ftb[b] = (int32_t)min(tb, (int64_t)INT32_MAX);
        a.lb[nlarge + (int32_t)((ex >> 32) & 0xffffu)] = b;
      } else if (small) {
        a.sl[nsmall + (int32_t)(ex >> 48)] = b;
      } else if (!direct) {
        a.d_nnz_y[b] = 0;
      }
    }
    tiles += (int64_t)(tot & 0xffffffffull);
    nlarge += (int32_t)((tot >> 32) & 0xffffu);
    nsmall += (int32_t)(tot >> 48);
  }
  // the direct frontiers: their tiles follow the large frontiers' tiles
  int64_t dtiles = 0;
  int32_t ndirect = 0;
  if (a.direct_min > 0) {
    for (int32_t base = 0; base < a.B; base += K6_THREADS) {
      const int32_t b = base + tid;
      const int32_t W = b < a.B ? __ldcg(a.fW + b) : 0;
      const bool direct = b < a.B && W > K6_SMALL_MAX && W >= a.direct_min;
      const unsigned long long T = direct ? (unsigned long long)(((int64_t)W + a.q - 1) / a.q) : 0ull;
      const unsigned long long v = T | ((unsigned long long)(direct ? 1 : 0) << 32);
      unsigned long long tot;
      const unsigned long long ex = block_exclusive_sum<K6_THREADS>(v, sh.scan, &tot);
      if (direct) {
        const int64_t tb = tiles + dtiles + (int64_t)(ex & 0xffffffffull);
        const int32_t di = ndirect + (int32_t)(ex >> 32);
        a.ftb[b] = (int32_t)min(tb, (int64_t)INT32_MAX);
        a.ld[di] = b;
        a.fdi[b] = di;
      }
      dtiles += (int64_t)(tot & 0xffffffffull);
      ndirect += (int32_t)(tot >> 32);
    }
  }
  if (tiles + dtiles > a.tiles_cap) {  // cannot happen with the host's bound; those frontiers are dropped
    if (tid == 0) atomicOr(a.status, ST_BOUND);
    tiles = 0;
    nlarge = 0;
    dtiles = 0;
    ndirect = 0;
  }
  const int32_t ndw = (ndirect + a.dslots - 1) / max(a.dslots, 1);
  __syncthreads();
  for (int32_t dw = tid; dw <= ndw && dw < a.dw_cap; dw += K6_THREADS)
    a.dwt0[dw] = dw < ndw ? __ldcg(a.ftb + __ldcg(a.ld + dw * a.dslots)) : (int32_t)(tiles + dtiles);
  __syncthreads();
  // waves: frontier b joins wave floor(first tile * q / win); a frontier's
  // padded products are at most win, so consecutive waves differ by one
  int32_t nw = 0;
  for (int32_t li = tid; li < nlarge; li += K6_THREADS) {
    const int32_t tb = __ldcg(a.ftb + __ldcg(a.lb + li));
    const int32_t w = (int32_t)((int64_t)tb * a.q / a.win);
    const int32_t wp = li == 0 ? -1 : (int32_t)((int64_t)__ldcg(a.ftb + __ldcg(a.lb + li - 1)) * a.q / a.win);
    if (w != wp && w < a.nw_cap) {
      a.wt0[w] = tb;
      a.wl0[w] = li;
    }
    if (li == nlarge - 1) sh.tot = w + 1;
  }
  __syncthreads();
  if (nlarge > 0) nw = sh.tot;
  if (nw > a.nw_cap) {
    if (tid == 0) atomicOr(a.status, ST_BOUND);
    nw = 0;
    nlarge = 0;
  }
  if (tid == 0) {
    a.wt0[nw] = (int32_t)tiles;
    a.wl0[nw] = nlarge;
    a.st->n_small = nsmall;
    a.st->n_large = nlarge;
    a.st->n_tiles = (int32_t)tiles;
    a.st->n_waves = nw;
    a.st->n_direct = ndirect;
    a.st->n_dwaves = ndw < a.dw_cap ? ndw : 0;
    if (ndw >= a.dw_cap && ndw > 0) atomicOr(a.status, ST_BOUND);
    a.st->padded = tiles * a.q;
  }
}

// ---------------------------------------------------------------------------
// phase 3: the first x entry of every tile of the large frontiers
// ---------------------------------------------------------------------------
__device__ void k6_tile_starts(const K6Args& a, int32_t n_large) {
  const int tid = threadIdx.x;
  for (int32_t c = blockIdx.x; c < a.nc; c += gridDim.x) {
    const int32_t b = k6_frontier_of_chunk(a.cp, a.B, c);
    const int32_t W = __ldcg(a.fW + b);
    if (W <= K6_SMALL_MAX) continue;
    const int32_t fc = __ldcg(a.ffc + b), xb = a.xp[b], tb = __ldcg(a.ftb + b);
    const int32_t e1 = min((c - a.cp[b] + 1) * K6_CH, fc);
    for (int32_t e = (c - a.cp[b]) * K6_CH + tid; e < e1; e += K6_THREADS) {
      const int32_t w = __ldcg(a.cw + xb + e);
      const int32_t wn = e + 1 < fc ? __ldcg(a.cw + xb + e + 1) : W;
      for (int32_t t = (int32_t)(((int64_t)w + a.q - 1) / a.q); (int64_t)t * a.q < wn; ++t) {
        if (tb + t >= a.tiles_cap) break;  // (the plan dropped the large frontiers)
        a.tk0[tb + t] = xb + e;
        a.tf[tb + t] = b;
      }
    }
  }
  const int64_t nst = (int64_t)n_large * a.nb;
  for (int64_t i = (int64_t)blockIdx.x * K6_THREADS + tid; i < nst; i += (int64_t)gridDim.x * K6_THREADS)
    a.bstat[i] = 0ull;
}

// ---------------------------------------------------------------------------
// phase 4a: a small frontier, whole, in one CTA
// ---------------------------------------------------------------------------
// Bitonic sorting network over n2 (a power of two) keys with their values.
__device__ void k6_bitonic(uint32_t* key, uint32_t* val, int n2) {
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < (n2 >> 1); i += K6_THREADS) {
        const int lo = ((i & ~(j - 1)) << 1) | (i & (j - 1));  // bit j of lo is 0
        const int hi = lo | j;
        const uint32_t ka = key[lo], kb = key[hi];
        if ((ka > kb) == ((lo & k) == 0)) {
          key[lo] = kb;
          key[hi] = ka;
          const uint32_t va = val[lo];
          val[lo] = val[hi];
          val[hi] = va;
        }
      }
      __syncthreads();
    }
  }
}

// The products of every x entry of a frontier with W <= QMAX products: the
// tile layout of the expand step (one tile), then sort by row, combine
// equal rows and write y_b.
template <int SEM>
__device__ void k6_small(const K6Args& a, int32_t b, unsigned char* smem, K6Shared& sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int32_t* kbase = (int32_t*)smem;
  uint32_t* kx = (uint32_t*)(kbase + QMAX + 1);
  uint32_t* hbits = kx + QMAX + 1;
  const int32_t W = __ldcg(a.fW + b), fc = __ldcg(a.ffc + b), xb = a.xp[b];
  for (int32_t l = tid; l < fc; l += K6_THREADS) {
    const int32_t w = __ldcg(a.cw + xb + l);
    kbase[l] = __ldcg(a.cb + xb + l) - w;
    kx[l] = __ldcg(a.cx + xb + l);
    if (l > 0 && w > 0 && w < W) atomicOr(&hbits[w >> 5], 1u << (w & 31));
  }
  __syncthreads();
  uint32_t rrow[K2_IMAX], rval[K2_IMAX];
  if (W == QMAX)
    k2_gather<SEM, K2_IMAX, true>(a.rowidx, a.val, hbits, kbase, kx, K2_IMAX, warp, lane, 0, W, a.nnz, rrow, rval);
  else
    k2_gather<SEM, K2_IMAX, false>(a.rowidx, a.val, hbits, kbase, kx, K2_IMAX, warp, lane, 0, W, a.nnz, rrow,
                                   rval);
  const uint32_t* mask = a.masks ? a.masks + (int64_t)b * a.mask_stride : nullptr;
#pragma unroll
  for (int i = 0; i < K2_IMAX; ++i) {
    const uint32_t row = rrow[i];
    if (row == 0xffffffffu) continue;
    if (row >= (uint32_t)a.m) {
      atomicOr(a.status, ST_INDEX);
      rrow[i] = 0xffffffffu;
    } else if (mask && ((__ldg(mask + (row >> 5)) >> (row & 31)) & 1u)) {
      rrow[i] = 0xffffffffu;  // complemented mask: a set bit removes the row
    }
  }
  __syncthreads();  // the x entries are read: their bytes take the keys and values
  for (int j = tid; j < QMAX / 32; j += K6_THREADS) hbits[j] = 0u;
  int n2 = 32;
  while (n2 < W) n2 <<= 1;
  uint32_t* skey = (uint32_t*)smem;
  uint32_t* sval = skey + QMAX;
#pragma unroll
  for (int i = 0; i < K2_IMAX; ++i) {
    const int p = warp * K2_IMAX * 32 + i * 32 + lane;  // the product this item holds
    if (p < n2) {
      skey[p] = rrow[i];
      sval[p] = rval[i];
    }
  }
  __syncthreads();
  k6_bitonic(skey, sval, n2);
  // thread tid owns positions [tid*per, tid*per + per); a head starts a run of one row
  const int per = n2 >= K6_THREADS ? n2 / K6_THREADS : 1;
  const int p0 = tid * per;
  uint32_t kk[K2_IMAX], vv[K2_IMAX];
  uint32_t heads = 0u;
#pragma unroll
  for (int i = 0; i < K2_IMAX; ++i) {
    kk[i] = 0xffffffffu;
    vv[i] = 0u;
    const int p = p0 + i;
    if (i < per && p < n2) {
      kk[i] = skey[p];
      vv[i] = sval[p];
      if (kk[i] != 0xffffffffu && (p == 0 || skey[p - 1] != kk[i])) heads |= 1u << i;
    }
  }
  int32_t nu;
  const int32_t ex = block_exclusive_sum<K6_THREADS>((int32_t)__popc(heads), sh.iscan, &nu);
  // the sorted keys are in registers: their bytes take the combined rows
  uint32_t* outk = skey;
  uint32_t* outv = sval;
  int32_t r = ex - 1;
#pragma unroll
  for (int i = 0; i < K2_IMAX; ++i) {
    if ((heads >> i) & 1u) {
      ++r;
      outk[r] = kk[i];
      outv[r] = sr_identity<SEM>();
    }
  }
  __syncthreads();
  if (SEM != kOrAnd) {
    r = ex - 1;
#pragma unroll
    for (int i = 0; i < K2_IMAX; ++i) {
      if ((heads >> i) & 1u) ++r;
      if (kk[i] != 0xffffffffu) spa_apply<SEM>(outv, (uint32_t)r, vv[i]);
    }
  }
  __syncthreads();
  const int32_t cap = a.y_cap[b];
  const int64_t yo = a.y_off[b];
  for (int32_t j = tid; j < nu && j < cap; j += K6_THREADS) {
    a.y_idx[yo + j] = (int32_t)outk[j];
    if (SEM != kOrAnd && a.y_val) a.y_val[yo + j] = outv[j];
  }
  if (tid == 0) {
    a.d_nnz_y[b] = nu;
    if (nu > cap) atomicOr(a.status, ST_CAPACITY);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// phase 4b: one tile of a large frontier (Step 1 into the tile's own slot)
// ---------------------------------------------------------------------------
template <int SEM, int IT>
__device__ void k6_tile(const K6Args& a, int32_t k, int32_t slot, unsigned char* smem, K6Shared& sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int32_t q = IT * K6_THREADS;
  int32_t* kbase = (int32_t*)smem;
  uint32_t* kx = (uint32_t*)(kbase + QMAX + 1);
  uint32_t* hbits = kx + QMAX + 1;
  int32_t* hist = (int32_t*)(hbits + QMAX / 32);
  uint32_t* hacc = (uint32_t*)(hist + a.nb + 1);  // the tile's hub sums
  int32_t* hrow = (int32_t*)(hacc + HOT_MAX);     // hub row ids (loaded when the phase starts)
  uint32_t* htb = (uint32_t*)(hrow + HOT_MAX);    // hubs the tile touched
  uint2* stage = (uint2*)smem;  // the staged products take the bytes of the x entries
  const int nb = a.nb, lwb = a.lwb;
  const int nhot = a.nhot;
  const uint32_t wmask = (1u << lwb) - 1u;
  const int32_t b = __ldcg(a.tf + k);
  const int32_t W = __ldcg(a.fW + b), fc = __ldcg(a.ffc + b), xb = a.xp[b], tb = __ldcg(a.ftb + b);
  const int32_t t = k - tb;
  const int32_t T = (int32_t)(((int64_t)W + q - 1) / q);
  const int32_t p0 = t * q;
  const int32_t np = min(q, W - p0);
  const int32_t e0 = __ldcg(a.tk0 + k);
  const int32_t e1 = t + 1 < T ? __ldcg(a.tk0 + k + 1) + 1 : xb + fc;
  const int32_t nk = max(1, min(e1 - e0, QMAX + 1));
  for (int32_t l = tid; l < nk; l += K6_THREADS) {
    const int32_t w = __ldcg(a.cw + e0 + l);
    kbase[l] = __ldcg(a.cb + e0 + l) - w;
    kx[l] = __ldcg(a.cx + e0 + l);
    const int32_t off = w - p0;
    if (l > 0 && off > 0 && off < np) atomicOr(&hbits[off >> 5], 1u << (off & 31));
  }
  for (int r = tid; r <= nb; r += K6_THREADS) hist[r] = 0;
  __syncthreads();
  uint32_t rrow[K2_IMAX], rval[K2_IMAX];
  int32_t rank[K2_IMAX];
  if (np == q)
    k2_gather<SEM, IT, true>(a.rowidx_t, a.val, hbits, kbase, kx, IT, warp, lane, p0, np, a.nnz, rrow, rval);
  else
    k2_gather<SEM, IT, false>(a.rowidx_t, a.val, hbits, kbase, kx, IT, warp, lane, p0, np, a.nnz, rrow, rval);
  const uint32_t* mask = a.masks ? a.masks + (int64_t)b * a.mask_stride : nullptr;
  const uint32_t masked = mask ? k2_mask_bits(mask, rrow, (uint32_t)a.m, (uint32_t)nhot, hrow) : 0u;
#pragma unroll
  for (int i = 0; i < K2_IMAX; ++i) {
    rank[i] = -1;
    const uint32_t row = rrow[i];
    if (row == 0xffffffffu) continue;
    if (row >= (uint32_t)a.m) {
      const uint32_t hs = row - (uint32_t)a.m;
      if (hs >= (uint32_t)nhot) {
        atomicOr(a.status, ST_INDEX);
        continue;
      }
      // a hub row: summed in the tile, staged once below
      if ((masked >> i) & 1u) continue;
      spa_apply<SEM>(hacc, hs, rval[i]);
      const uint32_t hb = 1u << (hs & 31);
      if (!(htb[hs >> 5] & hb)) atomicOr(&htb[hs >> 5], hb);
      continue;
    }
    if ((masked >> i) & 1u) continue;
    rank[i] = atomicAdd(&hist[row >> lwb], 1);
  }
  __syncthreads();
  for (int j = tid; j < QMAX / 32; j += K6_THREADS) hbits[j] = 0u;
  // every hub the tile touched is one more entry of its bucket
  constexpr int HPT = HOT_MAX / K6_THREADS;
  int32_t hrank[HPT];
#pragma unroll
  for (int k2 = 0; k2 < HPT; ++k2) {
    const int hs = tid + k2 * K6_THREADS;
    hrank[k2] = -1;
    if (hs < nhot && ((htb[hs >> 5] >> (hs & 31)) & 1u)) hrank[k2] = atomicAdd(&hist[hrow[hs] >> lwb], 1);
  }
  __syncthreads();
  // one warp turns the counts into the tile's bucket offsets
  if (warp == 0) {
    const int per = (nb + 31) >> 5;
    const int b0 = lane * per, b1 = min(b0 + per, nb);
    int32_t sum = 0;
    for (int r = b0; r < b1; ++r) sum += hist[r];
    int32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    int32_t run = x - sum;
    for (int r = b0; r < b1; ++r) {
      const int32_t c = hist[r];
      hist[r] = run;
      run += c;
    }
    if (lane == 31) {
      hist[nb] = x;
      sh.kept = x;
    }
  }
  __syncthreads();
  for (int r = tid; r <= nb; r += K6_THREADS) a.toff[(int64_t)r * a.tw + slot] = hist[r];
#pragma unroll
  for (int i = 0; i < K2_IMAX; ++i)
    if (rank[i] >= 0) stage[hist[rrow[i] >> lwb] + rank[i]] = make_uint2(rrow[i], rval[i]);
#pragma unroll
  for (int k2 = 0; k2 < HPT; ++k2) {
    const int hs = tid + k2 * K6_THREADS;
    if (hrank[k2] >= 0) {
      const uint32_t hr = (uint32_t)hrow[hs];
      stage[hist[hr >> lwb] + hrank[k2]] = make_uint2(hr, hacc[hs]);
      hacc[hs] = sr_identity<SEM>();  // untouched sums stay at the identity
    }
  }
  for (int j = tid; j < HOT_MAX / 32; j += K6_THREADS) htb[j] = 0u;
  __syncthreads();
  const int32_t kept = sh.kept;
  const int64_t dst0 = (int64_t)slot * q;
  for (int32_t s = tid; s < kept; s += K6_THREADS) {
    const uint2 e = stage[s];
    a.brow[dst0 + s] = (uint16_t)(e.x & wmask);
    if (SEM != kOrAnd) a.bval[dst0 + s] = e.y;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// direct form: one tile of a frontier with many products ((+,*), or
// (min, select2nd) with vertex ids as x values): every product applied to
// the frontier's accumulator in global memory (L2) with the semiring's add
// (a float reduction or an integer minimum), hub rows combined in the tile
// first
// ---------------------------------------------------------------------------
template <int SEM>
__device__ __forceinline__ void k6_acc_apply(uint32_t* acc, uint32_t r, uint32_t v) {
  if (SEM == kPlusTimes) atomicAdd(reinterpret_cast<float*>(acc) + r, __uint_as_float(v));
  else atomicMin(reinterpret_cast<int*>(acc) + r, (int)v);
}

template <int SEM, int IT>
__device__ void k6_tile_direct(const K6Args& a, int32_t k, uint32_t* acc, unsigned char* smem) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int32_t q = IT * K6_THREADS;
  int32_t* kbase = (int32_t*)smem;
  uint32_t* kx = (uint32_t*)(kbase + QMAX + 1);
  uint32_t* hbits = kx + QMAX + 1;
  int32_t* hist = (int32_t*)(hbits + QMAX / 32);
  uint32_t* hacc = (uint32_t*)(hist + a.nb + 1);
  int32_t* hrow = (int32_t*)(hacc + HOT_MAX);
  uint32_t* htb = (uint32_t*)(hrow + HOT_MAX);
  const int nhot = a.nhot;
  const int32_t b = __ldcg(a.tf + k);
  const int32_t W = __ldcg(a.fW + b), fc = __ldcg(a.ffc + b), xb = a.xp[b], tb = __ldcg(a.ftb + b);
  const int32_t t = k - tb;
  const int32_t T = (int32_t)(((int64_t)W + q - 1) / q);
  const int32_t p0 = t * q;
  const int32_t np = min(q, W - p0);
  const int32_t e0 = __ldcg(a.tk0 + k);
  const int32_t e1 = t + 1 < T ? __ldcg(a.tk0 + k + 1) + 1 : xb + fc;
  const int32_t nk = max(1, min(e1 - e0, QMAX + 1));
  for (int32_t l = tid; l < nk; l += K6_THREADS) {
    const int32_t w = __ldcg(a.cw + e0 + l);
    kbase[l] = __ldcg(a.cb + e0 + l) - w;
    kx[l] = __ldcg(a.cx + e0 + l);
    const int32_t off = w - p0;
    if (l > 0 && off > 0 && off < np) atomicOr(&hbits[off >> 5], 1u << (off & 31));
  }
  __syncthreads();
  uint32_t rrow[K2_IMAX], rval[K2_IMAX];
  if (np == q)
    k2_gather<SEM, IT, true>(a.rowidx_t, a.val, hbits, kbase, kx, IT, warp, lane, p0, np, a.nnz, rrow, rval);
  else
    k2_gather<SEM, IT, false>(a.rowidx_t, a.val, hbits, kbase, kx, IT, warp, lane, p0, np, a.nnz, rrow, rval);
  const uint32_t* mask = a.masks ? a.masks + (int64_t)b * a.mask_stride : nullptr;
  const uint32_t masked = mask ? k2_mask_bits(mask, rrow, (uint32_t)a.m, (uint32_t)nhot, hrow) : 0u;
#pragma unroll
  for (int i = 0; i < K2_IMAX; ++i) {
    const uint32_t row = rrow[i];
    if (row == 0xffffffffu) continue;
    if (row >= (uint32_t)a.m) {
      const uint32_t hs = row - (uint32_t)a.m;
      if (hs >= (uint32_t)nhot) {
        atomicOr(a.status, ST_INDEX);
        continue;
      }
      if ((masked >> i) & 1u) continue;
      spa_apply<SEM>(hacc, hs, rval[i]);
      const uint32_t hb = 1u << (hs & 31);
      if (!(htb[hs >> 5] & hb)) atomicOr(&htb[hs >> 5], hb);
      continue;
    }
    if ((masked >> i) & 1u) continue;
    k6_acc_apply<SEM>(acc, row, rval[i]);
  }
  __syncthreads();
  for (int j = tid; j < QMAX / 32; j += K6_THREADS) hbits[j] = 0u;
  for (int hs = tid; hs < nhot; hs += K6_THREADS) {
    if ((htb[hs >> 5] >> (hs & 31)) & 1u) {
      k6_acc_apply<SEM>(acc, (uint32_t)hrow[hs], hacc[hs]);
      hacc[hs] = sr_identity<SEM>();
    }
  }
  __syncthreads();
  for (int j = tid; j < HOT_MAX / 32; j += K6_THREADS) htb[j] = 0u;
  __syncthreads();
}

// The direct form's compaction: row tile rt (K6_DROWS rows) of one
// frontier's accumulator, its touched rows (not the empty mark: -0.0 for
// (+,*), INT32_MAX for (min, select2nd)) to y_b in ascending order, each
// reset to the mark; the tile's offset in y_b from a look-back along the
// frontier's row tiles.
constexpr int K6_DSTEPS = 16;                           // 32-row words per warp and tile
constexpr int K6_DROWS = K6_THREADS * K6_DSTEPS;        // rows per tile (8192)

template <int SEM>
__device__ void k6_dcompact(const K6Args& a, int32_t b, uint32_t* acc, unsigned long long* chain, int32_t rt,
                            K6Shared& sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t kEmpty = spa_empty<SEM>();
  const int64_t r0 = (int64_t)rt * K6_DROWS + (int64_t)warp * (K6_DSTEPS * 32) + lane;
  uint32_t v[K6_DSTEPS], bits[K6_DSTEPS];
  int32_t cw = 0;
#pragma unroll
  for (int k = 0; k < K6_DSTEPS; ++k) v[k] = r0 + k * 32 < a.m ? __ldcg(acc + r0 + k * 32) : kEmpty;
#pragma unroll
  for (int k = 0; k < K6_DSTEPS; ++k) {
    bits[k] = __ballot_sync(0xffffffffu, v[k] != kEmpty);
    cw += __popc(bits[k]);
  }
  int32_t tot;
  const int32_t run = block_exclusive_sum<K6_THREADS>(lane == 0 ? cw : 0, sh.iscan, &tot);
  if (tid < 32) {
    const unsigned long long pre = warp_lookback(chain, (uint32_t)rt, (unsigned long long)tot, a.status);
    if (tid == 0) sh.off = (long long)pre;
  }
  __syncthreads();
  const int32_t cap = a.y_cap[b];
  const int64_t yo = a.y_off[b];
  const uint32_t lt = (1u << lane) - 1u;
  int64_t pos = sh.off + __shfl_sync(0xffffffffu, run, 0);
#pragma unroll
  for (int k = 0; k < K6_DSTEPS; ++k) {
    if ((bits[k] >> lane) & 1u) {
      const int64_t r = r0 + k * 32;
      const int64_t pp = pos + __popc(bits[k] & lt);
      if (pp < cap) {
        a.y_idx[yo + pp] = (int32_t)r;
        if (a.y_val) a.y_val[yo + pp] = v[k];
      }
      acc[r] = kEmpty;
    }
    pos += __popc(bits[k]);
  }
  if (rt == a.nrt - 1 && tid == 0) {
    const int64_t total = sh.off + tot;
    a.d_nnz_y[b] = (int32_t)total;
    if (total > cap) atomicOr(a.status, ST_CAPACITY);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// phase 5: one (frontier, bucket) merge task
// ---------------------------------------------------------------------------
template <int SEM>
__device__ void k6_merge(const K6Args& a, int32_t li, int r, int32_t wt0w, unsigned char* smem, K6Shared& sh) {
  // dense SPA: (+,*) marks empty rows with -0.0; (min, select2nd) with
  // INT32_MAX when the x values are vertex ids (no product can carry it)
  const bool kDenseForm = SEM == kPlusTimes || (SEM == kMinSelect2nd && a.x_ids);
  constexpr int U = 4;  // units of 32 four-entry chunks a warp reads at once
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int lwb = a.lwb;
  const int32_t wb = 1 << lwb;
  const uint32_t wmask = (uint32_t)wb - 1u;
  const int nw = wb >> 5;
  uint32_t* spa = (uint32_t*)smem;
  uint32_t* occ = spa + wb;
  int32_t* seg_lo = (int32_t*)(occ + nw);
  int32_t* seg_n = seg_lo + K6_SEGMAX;
  int32_t* seg_u = seg_n + K6_SEGMAX;  // [K6_SEGMAX + 1]
  const int32_t b = __ldcg(a.lb + li);
  const int32_t W = __ldcg(a.fW + b), tb = __ldcg(a.ftb + b);
  const int32_t q = a.q;
  const int32_t T = (int32_t)(((int64_t)W + q - 1) / q);
  const int32_t s0 = tb - wt0w;  // the frontier's first tile slot in this wave
  const int32_t* offA = a.toff + (int64_t)r * a.tw + s0;
  const int32_t* offB = offA + a.tw;
  // the bucket's run in every tile of the frontier (listed while it fits)
  int32_t c = 0;
  for (int32_t j = tid; j < T; j += K6_THREADS) {
    const int32_t lo = __ldcg(offA + j), hi = __ldcg(offB + j);
    if (j < K6_SEGMAX) {
      seg_lo[j] = lo;
      seg_n[j] = hi - lo;
    }
    c += hi - lo;
  }
  int32_t cnt;
  block_exclusive_sum<K6_THREADS>(c, sh.iscan, &cnt);
  const bool active = cnt > 0;
  const bool dense = kDenseForm && wb >= K6_DENSE_MIN_WB && (int64_t)cnt * K6_DENSE_DIV >= wb;
  const uint32_t ident = sr_identity<SEM>();
  const uint32_t empty = spa_empty<SEM>();
  if (active) {
    if (dense) {
      uint4* s4 = reinterpret_cast<uint4*>(spa);
      for (int i = tid; i < (wb >> 2); i += K6_THREADS) s4[i] = make_uint4(empty, empty, empty, empty);
    } else {
      for (int w = tid; w < nw; w += K6_THREADS) occ[w] = 0u;
      if (SEM != kOrAnd) {
        if ((int64_t)cnt * 16 < wb && T <= K6_SEGMAX) {
          // partial initialisation: only the slots this bucket touches (Sec. II-F)
          for (int32_t j = warp; j < T; j += K6_WARPS) {
            const int64_t base = (int64_t)(s0 + j) * q + seg_lo[j];
            for (int32_t e = lane; e < seg_n[j]; e += 32) spa[__ldcg(a.brow + base + e) & wmask] = ident;
          }
        } else {
          for (int i = tid; i < wb; i += K6_THREADS) spa[i] = ident;
        }
      }
    }
    __syncthreads();
    // Step 2: the runs into the SPA.  A run is cut into 32-entry units (one
    // per warp step); a warp takes a contiguous range of the units, U at a
    // time with all their loads in flight, following the run list forward.
    for (int32_t j0 = 0; j0 < T; j0 += K6_SEGMAX) {
      const int32_t ns = min(K6_SEGMAX, T - j0);
      if (j0 > 0) {
        __syncthreads();
        for (int32_t j = tid; j < ns; j += K6_THREADS) {
          const int32_t lo = __ldcg(offA + j0 + j), hi = __ldcg(offB + j0 + j);
          seg_lo[j] = lo;
          seg_n[j] = hi - lo;
        }
        __syncthreads();
      }
      // units before each run (seg_u[ns] = all units of this part of the
      // list); a unit is 32 aligned 4-entry chunks of one run, one per lane
      {
        constexpr int SPT = K6_SEGMAX / K6_THREADS;
        int32_t uc[SPT], tsum = 0;
#pragma unroll
        for (int i = 0; i < SPT; ++i) {
          const int32_t j = tid * SPT + i;
          uc[i] = 0;
          if (j < ns && seg_n[j] > 0) {
            const int32_t chunks = ((seg_lo[j] + seg_n[j] + 3) >> 2) - (seg_lo[j] >> 2);
            uc[i] = (chunks + 31) >> 5;
          }
          tsum += uc[i];
        }
        int32_t nu;
        int32_t ex = block_exclusive_sum<K6_THREADS>(tsum, sh.iscan, &nu);
#pragma unroll
        for (int i = 0; i < SPT; ++i) {
          const int32_t j = tid * SPT + i;
          if (j < ns) seg_u[j] = ex;
          ex += uc[i];
        }
        if (tid == 0) seg_u[ns] = nu;
        __syncthreads();
      }
      const int32_t nu = seg_u[ns];
      const int32_t per = (nu + K6_WARPS - 1) / K6_WARPS;
      const int32_t u_end = min(nu, (warp + 1) * per);
      int32_t u = warp * per;
      int32_t j = 0;
      if (u < u_end) {  // the run holding unit u: the last j with seg_u[j] <= u
        int32_t lo = 0, hi = ns - 1;
        while (lo < hi) {
          const int32_t mid = (lo + hi + 1) >> 1;
          if (seg_u[mid] <= u) lo = mid;
          else hi = mid - 1;
        }
        j = lo;
      }
      const uint2* brow4 = reinterpret_cast<const uint2*>(a.brow);  // 4 row offsets
      const uint4* bval4 = reinterpret_cast<const uint4*>(a.bval);  // 4 values
      for (; u < u_end; u += U) {
        uint2 rr[U];
        uint4 vv[U];
        int32_t e0[U], ea[U], eb[U];  // the chunk's first entry, the run's entries [ea, eb)
#pragma unroll
        for (int k = 0; k < U; ++k) {
          const int32_t uu = u + k;
          rr[k] = make_uint2(0u, 0u);
          vv[k] = make_uint4(0u, 0u, 0u, 0u);
          e0[k] = 0;
          ea[k] = 0;
          eb[k] = 0;
          if (uu < u_end) {
            while (seg_u[j + 1] <= uu) ++j;
            const int32_t lo = seg_lo[j], hi = lo + seg_n[j];
            const int32_t c = (lo >> 2) + ((uu - seg_u[j]) << 5) + lane;  // chunk inside the tile slot
            if (c < ((hi + 3) >> 2)) {
              const int64_t base = (int64_t)(s0 + j0 + j) * q + 4 * c;  // a multiple of 4
              rr[k] = __ldcg(brow4 + (base >> 2));
              if (SEM != kOrAnd) vv[k] = __ldcg(bval4 + (base >> 2));
              e0[k] = 4 * c;
              ea[k] = lo;
              eb[k] = hi;
            }
          }
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
          const uint32_t rw[4] = {rr[k].x & 0xffffu, rr[k].x >> 16, rr[k].y & 0xffffu, rr[k].y >> 16};
          const uint32_t vw[4] = {vv[k].x, vv[k].y, vv[k].z, vv[k].w};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int32_t e = e0[k] + t;
            if (e < ea[k] || e >= eb[k]) continue;
            const uint32_t x = rw[t] & wmask;
            if (!dense) atomicOr(occ + (x >> 5), 1u << (x & 31));
            spa_apply<SEM>(spa, x, vw[t]);
          }
        }
      }
    }
    __syncthreads();
  }
  // Step 3: the bucket's unique rows, its offset in y_b, its rows in order
  const int rpw = wb / K6_WARPS;
  const int wpt = nw > K6_THREADS ? nw / K6_THREADS : 1;
  const int w0 = tid * wpt;
  int32_t cu = 0;
  if (dense) {
    int32_t cwp = 0;
    for (int i = warp * rpw + lane; i < (warp + 1) * rpw; i += 32)
      cwp += __popc(__ballot_sync(0xffffffffu, spa[i] != empty));
    cu = lane == 0 ? cwp : 0;
  } else if (active && w0 < nw) {
    for (int w = w0; w < w0 + wpt; ++w) cu += __popc(occ[w]);
  }
  int32_t tot;
  const int32_t run = block_exclusive_sum<K6_THREADS>(cu, sh.iscan, &tot);
  if (tid < 32) {
    const unsigned long long pre =
        warp_lookback(a.bstat + (int64_t)li * a.nb, (uint32_t)r, (unsigned long long)tot, a.status);
    if (tid == 0) sh.off = (long long)pre;
  }
  __syncthreads();
  const int64_t off = sh.off;
  const int32_t cap = a.y_cap[b];
  const int64_t yo = a.y_off[b];
  const int32_t row0 = r << lwb;
  if (dense) {
    int64_t pos = off + __shfl_sync(0xffffffffu, run, 0);
    const uint32_t lt = (1u << lane) - 1u;
    for (int r0w = warp * rpw; r0w < (warp + 1) * rpw; r0w += 32) {
      const uint32_t v = spa[r0w + lane];
      const bool hit = v != empty;
      const uint32_t bits = __ballot_sync(0xffffffffu, hit);
      if (hit) {
        const int64_t p = pos + __popc(bits & lt);
        if (p < cap) {
          a.y_idx[yo + p] = row0 + r0w + lane;
          if (a.y_val) a.y_val[yo + p] = v;
        }
      }
      pos += __popc(bits);
    }
  } else if (active && w0 < nw) {
    int64_t pos = off + run;
    for (int w = w0; w < w0 + wpt; ++w) {
      uint32_t bits = occ[w];
      while (bits) {
        const int i = (w << 5) + __ffs(bits) - 1;
        bits &= bits - 1u;
        if (pos < cap) {
          a.y_idx[yo + pos] = row0 + i;
          if (SEM != kOrAnd && a.y_val) a.y_val[yo + pos] = spa[i];
        }
        ++pos;
      }
    }
  }
  if (r == a.nb - 1 && tid == 0) {
    const int64_t total = off + tot;
    a.d_nnz_y[b] = (int32_t)total;
    if (total > cap) atomicOr(a.status, ST_CAPACITY);
  }
  __syncthreads();
}

// The expand phase's shared state at its start: no entry starts marked, the
// hub table loaded, the hub sums at the semiring's identity.
template <int SEM>
__device__ void k6_expand_setup(const K6Args& a, unsigned char* smem) {
  const int tid = threadIdx.x;
  uint32_t* hbits = (uint32_t*)(smem + sizeof(int32_t) * 2 * (QMAX + 1));
  int32_t* hist = (int32_t*)(hbits + QMAX / 32);
  uint32_t* hacc = (uint32_t*)(hist + a.nb + 1);
  int32_t* hrow = (int32_t*)(hacc + HOT_MAX);
  uint32_t* htb = (uint32_t*)(hrow + HOT_MAX);
  for (int j = tid; j < QMAX / 32; j += K6_THREADS) hbits[j] = 0u;
  for (int h = tid; h < HOT_MAX; h += K6_THREADS) {
    hacc[h] = sr_identity<SEM>();
    hrow[h] = h < a.nhot ? a.hot_rows[h] : 0;
  }
  for (int j = tid; j < HOT_MAX / 32; j += K6_THREADS) htb[j] = 0u;
  __syncthreads();
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------
template <int SEM, int IT>
__global__ void __launch_bounds__(K6_THREADS, 2) k6_batched(K6Args a) {
  extern __shared__ __align__(16) unsigned char k6_smem_raw[];
  __shared__ K6Shared sh;
  const int tid = threadIdx.x;
  uint32_t epoch = 0;
  if (blockIdx.x == 0 && tid == 0) a.st->t[0] = k6_clock();
  k6_scan(a, k6_smem_raw, sh);
  if (!k6_barrier(a, ++epoch, sh)) return;
  if (blockIdx.x == 0) k6_plan(a, sh);
  if (!k6_barrier(a, ++epoch, sh)) return;
  const int32_t n_waves = __ldcg(&a.st->n_waves);
  const int32_t n_small = __ldcg(&a.st->n_small);
  const int32_t n_large = __ldcg(&a.st->n_large);
  k6_tile_starts(a, n_large);
  if (!k6_barrier(a, ++epoch, sh)) return;
  k6_expand_setup<SEM>(a, k6_smem_raw);
  if (SEM != kOrAnd) {
    // the direct frontiers, dslots at a time: every tile's products into the
    // frontier's accumulator, then the accumulators compacted into y (none
    // unless the host enabled the form)
    const int32_t n_direct = __ldcg(&a.st->n_direct);
    const int32_t n_dw = __ldcg(&a.st->n_dwaves);
    for (int dw = 0; dw < n_dw; ++dw) {
      const int32_t d0 = dw * a.dslots;
      const int32_t nd = min(a.dslots, n_direct - d0);
      const int32_t t0 = __ldcg(a.dwt0 + dw), t1 = __ldcg(a.dwt0 + dw + 1);
      for (int64_t i = (int64_t)blockIdx.x * K6_THREADS + tid; i < (int64_t)nd * a.nrt;
           i += (int64_t)gridDim.x * K6_THREADS)
        a.dstat[i] = 0ull;
      uint32_t* tkd = a.tk + 2 * (a.nw_cap + dw);
      for (;;) {
        if (tid == 0) sh.item = atomicAdd(tkd, 1u);
        __syncthreads();
        const uint32_t it = sh.item;
        if (it >= (uint32_t)(t1 - t0)) break;
        const int32_t k = t0 + (int32_t)it;
        const int32_t slot = __ldcg(a.fdi + __ldcg(a.tf + k)) - d0;
        k6_tile_direct<SEM, IT>(a, k, a.dacc + (int64_t)slot * a.m, k6_smem_raw);
      }
      if (!k6_barrier(a, ++epoch, sh)) return;
      // compaction tasks go tile-major: row tile rt of every frontier of the wave, then rt+1
      const uint32_t tasks = (uint32_t)(nd * a.nrt);
      for (;;) {
        if (tid == 0) sh.item = atomicAdd(tkd + 1, 1u);
        __syncthreads();
        const uint32_t g = sh.item;
        if (g >= tasks) break;
        const int32_t slot = (int32_t)(g % (uint32_t)nd), rt = (int32_t)(g / (uint32_t)nd);
        const int32_t b = __ldcg(a.ld + d0 + slot);
        k6_dcompact<SEM>(a, b, a.dacc + (int64_t)slot * a.m, a.dstat + (int64_t)slot * a.nrt, rt, sh);
      }
      if (!k6_barrier(a, ++epoch, sh)) return;
    }
  }
  const int passes = n_waves > 0 ? n_waves : 1;
  for (int w = 0; w < passes; ++w) {
    const int32_t t0 = w < n_waves ? __ldcg(a.wt0 + w) : 0;
    const int32_t t1 = w < n_waves ? __ldcg(a.wt0 + w + 1) : 0;
    const int32_t ns = w == 0 ? n_small : 0;
    const uint32_t items = (uint32_t)(ns + (t1 - t0));
    for (;;) {
      if (tid == 0) sh.item = atomicAdd(a.tk + 2 * w, 1u);
      __syncthreads();
      const uint32_t it = sh.item;
      if (it >= items) break;
      if ((int32_t)it < ns) k6_small<SEM>(a, __ldcg(a.sl + it), k6_smem_raw, sh);
      else k6_tile<SEM, IT>(a, t0 + (int32_t)it - ns, (int32_t)it - ns, k6_smem_raw, sh);
    }
    if (w >= n_waves) break;  // no large frontier
    if (!k6_barrier(a, ++epoch, sh)) return;
    // tasks go bucket-major (bucket r of every frontier of the wave, then r+1):
    // the bucket before a task in its frontier's look-back chain was handed
    // out one round earlier and is mostly done when the task needs its count
    const int32_t l0 = __ldcg(a.wl0 + w), l1 = __ldcg(a.wl0 + w + 1);
    const uint32_t nl = (uint32_t)(l1 - l0);
    const uint32_t tasks = nl * (uint32_t)a.nb;
    for (;;) {
      if (tid == 0) sh.item = atomicAdd(a.tk + 2 * w + 1, 1u);
      __syncthreads();
      const uint32_t g = sh.item;
      if (g >= tasks) break;
      k6_merge<SEM>(a, l0 + (int32_t)(g % nl), (int)(g / nl), t0, k6_smem_raw, sh);
    }
    if (w + 1 < passes) {
      if (!k6_barrier(a, ++epoch, sh)) return;
      k6_expand_setup<SEM>(a, k6_smem_raw);
    }
  }
  if (tid == 0) atomicMax(&a.st->t[K6_STAMPS - 1], k6_clock());
}

// Largest column length (bounds a frontier's tiles on the host).
__global__ void k6_max_col(const int32_t* __restrict__ colptr, int32_t ncols, int32_t* __restrict__ out) {
  int32_t mx = 0;
  for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < ncols; j += gridDim.x * blockDim.x)
    mx = max(mx, colptr[j + 1] - colptr[j]);
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

// A device array that only grows (its contents are not kept).
template <typename T>
struct DevArr {
  T* p = nullptr;
  size_t cap = 0;
  cudaError_t grow(size_t need) {
    if (need <= cap && p) return cudaSuccess;
    cudaFree(p);
    p = nullptr;
    cap = 0;
    const size_t n = std::max<size_t>(need, 1);
    cudaError_t e = cudaMalloc(&p, sizeof(T) * n);
    if (e == cudaSuccess) cap = n;
    return e;
  }
  void release() {
    cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

}  // namespace

struct K6Buffers {
  DevArr<K6State> st;
  DevArr<uint32_t> tk;
  DevArr<int32_t> wt0, wl0;
  DevArr<unsigned long long> cstat;
  DevArr<int32_t> xp, cp, fW, ffc, ftb, lb, sl;
  DevArr<int32_t> cw, cb;
  DevArr<uint32_t> cx;
  DevArr<int32_t> tk0, tf;
  DevArr<uint16_t> brow;
  DevArr<uint32_t> bval;
  DevArr<int32_t> toff;
  DevArr<unsigned long long> bstat;
  DevArr<uint32_t> dacc;            // direct accumulators, the mark dacc_empty in every row between launches
  uint32_t dacc_empty = 0u;
  DevArr<unsigned long long> dstat;
  DevArr<int32_t> ld, fdi, dwt0;
  int32_t* h_pin = nullptr;       // pinned: x_cnt[B] | xp[B+1] | cp[B+1]
  size_t cap_pin = 0;
  long long* h_padded = nullptr;  // pinned: the padded products of the last launch
  cudaEvent_t uploaded = nullptr; // the last upload from h_pin
  int uploaded_valid = 0;
  int32_t maxcol = -1;            // the matrix's largest column
  size_t smem_set[3][2] = {};     // dynamic shared memory each kernel variant is allowed
};

namespace {

int ceil_log2_i64(int64_t v) {
  int k = 0;
  while (((int64_t)1 << k) < v) ++k;
  return k;
}

template <int SEM, int IT>
cudaError_t k6_launch(K6Buffers* kb, const K6Args& a, size_t smem, int sm_count, cudaStream_t s) {
  auto fn = k6_batched<SEM, IT>;
  size_t& allowed = kb->smem_set[SEM][IT == K2_IMAX ? 1 : 0];
  if (allowed < smem) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    allowed = smem;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, K6_THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(std::min(per_sm, 2) * sm_count));
  cfg.blockDim = dim3(K6_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, a);
}

}  // namespace

void release_k6(spmspv_handle* h) {
  K6Buffers* kb = (K6Buffers*)h->k6;
  if (!kb) return;
  kb->st.release();
  kb->tk.release();
  kb->wt0.release();
  kb->wl0.release();
  kb->cstat.release();
  kb->xp.release();
  kb->cp.release();
  kb->fW.release();
  kb->ffc.release();
  kb->ftb.release();
  kb->lb.release();
  kb->sl.release();
  kb->cw.release();
  kb->cb.release();
  kb->cx.release();
  kb->tk0.release();
  kb->tf.release();
  kb->brow.release();
  kb->bval.release();
  kb->toff.release();
  kb->bstat.release();
  kb->dacc.release();
  kb->dstat.release();
  kb->ld.release();
  kb->fdi.release();
  kb->dwt0.release();
  cudaFreeHost(kb->h_pin);
  cudaFreeHost(kb->h_padded);
  if (kb->uploaded) cudaEventDestroy(kb->uploaded);
  delete kb;
  h->k6 = nullptr;
}

// One batched step as a single persistent launch (see the top of this file).
// x_cnt is read on the host first (one synchronisation of `s`) to size the
// work arrays.
int run_batched_k6(spmspv_handle* h, int sem, int32_t B, const int32_t* x_off, const int32_t* x_cnt,
                   const int32_t* x_idx, const uint32_t* x_val, const uint32_t* masks, int64_t mask_stride,
                   uint32_t opts, const int32_t* y_off, const int32_t* y_cap, int32_t* y_idx, uint32_t* y_val,
                   int32_t* d_nnz_y, cudaStream_t s, bool x_ids) {
  if (!h->k6) h->k6 = new K6Buffers();
  K6Buffers* kb = (K6Buffers*)h->k6;
  const Matrix& A = h->A;
  int sid = h->default_sched;
  if (opts & SPMSPV_SCHED_FORCE) sid = (int)SPMSPV_SCHED_ID(opts);
  if (sid >= SPMSPV_NUM_SCHEDULES / 2) sid -= SPMSPV_NUM_SCHEDULES / 2;  // the push form
  const Sched sc = decode_schedule(h, sid);
  const int q = sc.q;
  // bucket rows: m/256, m/128 or m/64 by the schedule's width (a tile's run of
  // one bucket is then q/nb products on average), at most 2^15 rows
  int lwb = ceil_log2_i64(A.m) - 8 + sid % 3;
  lwb = std::min(std::max(lwb, LWB_MIN), LWB_MAX);
  const int nb = (int)(((int64_t)A.m + (1 << lwb) - 1) >> lwb);
  if (nb > K6_NB_MAX) return fail(SPMSPV_ERR_UNSUPPORTED, "too many rows for the batched form (m = %d)", A.m);
  cudaError_t e;
  // pinned staging: x_cnt, then the two prefix arrays
  const size_t need_pin = (size_t)B * 3 + 2;
  if (kb->uploaded_valid) {  // the previous call's upload has left the staging buffer
    if ((e = cudaEventSynchronize(kb->uploaded)) != cudaSuccess) return cuda_fail(e, "batched staging");
    kb->uploaded_valid = 0;
  }
  if (kb->cap_pin < need_pin) {
    cudaFreeHost(kb->h_pin);
    kb->h_pin = nullptr;
    kb->cap_pin = 0;
    if ((e = cudaMallocHost(&kb->h_pin, sizeof(int32_t) * need_pin)) != cudaSuccess)
      return cuda_fail(e, "batched staging");
    kb->cap_pin = need_pin;
  }
  if (!kb->h_padded) {
    if ((e = cudaMallocHost(&kb->h_padded, sizeof(long long))) != cudaSuccess)
      return cuda_fail(e, "batched staging");
    *kb->h_padded = 0;
  }
  if (!kb->uploaded && (e = cudaEventCreateWithFlags(&kb->uploaded, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(e, "batched event");
  if (kb->maxcol < 0) {
    DevArr<int32_t> d;
    if ((e = d.grow(1)) != cudaSuccess) return cuda_fail(e, "batched max column");
    cudaMemsetAsync(d.p, 0, sizeof(int32_t), s);
    const int32_t ncols = A.jc ? A.nzc : A.n;
    if (ncols > 0) k6_max_col<<<h->sm_count * 2, 256, 0, s>>>(A.colptr, ncols, d.p);
    int32_t mc = 0;
    cudaMemcpyAsync(&mc, d.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
    d.release();
    if (e != cudaSuccess) return cuda_fail(e, "batched max column");
    kb->maxcol = mc;
  }
  int32_t* hc = kb->h_pin;
  cudaMemcpyAsync(hc, x_cnt, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, s);
  if (kb->st.p) cudaMemcpyAsync(kb->h_padded, &kb->st.p->padded, sizeof(long long), cudaMemcpyDeviceToHost, s);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "batched counts");
  // prefixes over the frontiers and the bounds of this call
  int32_t* hxp = hc + B;
  int32_t* hcp = hxp + B + 1;
  int64_t F = 0, nc = 0, tiles = 1;
  for (int32_t b = 0; b < B; ++b) {
    const int64_t c = hc[b];
    if (c < 0 || c > A.n) return fail(SPMSPV_ERR_ARG, "x_cnt[%d] = %lld outside [0, n]", b, (long long)c);
    hxp[b] = (int32_t)F;
    hcp[b] = (int32_t)nc;
    F += c;
    nc += (c + K6_CH - 1) / K6_CH;
    const int64_t wmax = std::min<int64_t>(A.nnz, c * (int64_t)kb->maxcol);
    tiles += (wmax + QF - 1) / QF;
    if (F >= INT32_MAX || nc >= INT32_MAX || tiles >= INT32_MAX)
      return fail(SPMSPV_ERR_UNSUPPORTED, "batch too large for one launch");
  }
  hxp[B] = (int32_t)F;
  hcp[B] = (int32_t)nc;
  if (F == 0) {
    if ((e = cudaMemsetAsync(d_nnz_y, 0, sizeof(int32_t) * B, s)) != cudaSuccess) return cuda_fail(e, "batched");
    h->last_stream = s;
    return SPMSPV_OK;
  }
  // wave window: the last launch's padded products (a repeated batch then
  // runs in one wave), at least one whole frontier, at most 2^28 entries
  const int64_t one = A.nnz + 4096;
  int64_t win = std::max<int64_t>(one, std::min<int64_t>(*kb->h_padded + 4096, (int64_t)1 << 28));
  win = (win + 4095) / 4096 * 4096;
  const int64_t capw = win + one + 4096;
  const int64_t tw = capw / QF + 1;
  // a frontier's padded products are at most 2048 * (its 2048-product tiles + 2)
  const int64_t nw_cap = (tiles + 2 * (int64_t)B) * QF / win + 2;
  // direct form ((+,*), m <= 2^24): frontiers with at least m/2 products, as
  // many per wave as accumulators fit in 128 MB (at most 32; measured on the
  // 256-frontier R-MAT s20 batch: 64 MB 1.116 ms, 128 MB 1.093 ms; a
  // threshold of m/4 or m instead of m/2: 1.102 / 1.159 ms)
  // (min, select2nd) takes the direct form when the x values are vertex ids
  // (INT32_MAX then marks an untouched row)
  const bool direct = (sem == kPlusTimes || (sem == kMinSelect2nd && x_ids)) && !(opts & SPMSPV_BUCKETS_ONLY) &&
                      A.m <= DIRECT_M_MAX;
  const int32_t dslots = direct ? (int32_t)std::max<int64_t>(1, std::min<int64_t>(32, ((int64_t)128 << 20) /
                                                                                   (4 * (int64_t)A.m)))
                                : 1;
  const int32_t nrt = (int32_t)(((int64_t)A.m + K6_DROWS - 1) / K6_DROWS);
  const int64_t dw_cap = (int64_t)B + 2;
  if (direct) {
    // every row of the accumulators holds the semiring's empty mark between
    // launches (the compaction restores it): new accumulators, and those
    // last used by the other semiring, are filled first
    const uint32_t empty = sem == kPlusTimes ? 0x80000000u : 0x7fffffffu;
    const bool grown = kb->dacc.cap < (size_t)dslots * A.m;
    if (grown && (e = kb->dacc.grow((size_t)dslots * A.m)) != cudaSuccess) {
      cudaGetLastError();
      return fail(SPMSPV_ERR_OOM, "batched accumulators: %s", cudaGetErrorString(e));
    }
    if (grown || kb->dacc_empty != empty) {
      if ((e = launch_fill_u32(kb->dacc.p, (int64_t)kb->dacc.cap, empty, s)) != cudaSuccess)
        return cuda_fail(e, "batched accumulators");
      kb->dacc_empty = empty;
    }
  }
  if ((e = kb->dstat.grow((size_t)dslots * nrt)) != cudaSuccess || (e = kb->ld.grow((size_t)B)) != cudaSuccess ||
      (e = kb->fdi.grow((size_t)B)) != cudaSuccess || (e = kb->dwt0.grow((size_t)dw_cap)) != cudaSuccess) {
    cudaGetLastError();
    return fail(SPMSPV_ERR_OOM, "batched work arrays: %s", cudaGetErrorString(e));
  }
  if ((e = kb->st.grow(1)) != cudaSuccess || (e = kb->tk.grow((size_t)(nw_cap + dw_cap) * 2)) != cudaSuccess ||
      (e = kb->wt0.grow((size_t)nw_cap + 1)) != cudaSuccess || (e = kb->wl0.grow((size_t)nw_cap + 1)) != cudaSuccess ||
      (e = kb->cstat.grow((size_t)nc)) != cudaSuccess || (e = kb->xp.grow((size_t)B + 1)) != cudaSuccess ||
      (e = kb->cp.grow((size_t)B + 1)) != cudaSuccess || (e = kb->fW.grow((size_t)B)) != cudaSuccess ||
      (e = kb->ffc.grow((size_t)B)) != cudaSuccess || (e = kb->ftb.grow((size_t)B)) != cudaSuccess ||
      (e = kb->lb.grow((size_t)B)) != cudaSuccess || (e = kb->sl.grow((size_t)B)) != cudaSuccess ||
      (e = kb->cw.grow((size_t)F)) != cudaSuccess || (e = kb->cb.grow((size_t)F)) != cudaSuccess ||
      (e = kb->cx.grow((size_t)F)) != cudaSuccess || (e = kb->tk0.grow((size_t)tiles)) != cudaSuccess ||
      (e = kb->tf.grow((size_t)tiles)) != cudaSuccess || (e = kb->brow.grow((size_t)capw)) != cudaSuccess ||
      (e = kb->bval.grow((size_t)capw)) != cudaSuccess ||
      (e = kb->toff.grow((size_t)(nb + 1) * (size_t)tw)) != cudaSuccess ||
      (e = kb->bstat.grow((size_t)B * nb)) != cudaSuccess) {
    cudaGetLastError();
    return fail(SPMSPV_ERR_OOM, "batched work arrays: %s", cudaGetErrorString(e));
  }
  cudaMemcpyAsync(kb->xp.p, hxp, sizeof(int32_t) * (B + 1), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(kb->cp.p, hcp, sizeof(int32_t) * (B + 1), cudaMemcpyHostToDevice, s);
  cudaEventRecord(kb->uploaded, s);
  kb->uploaded_valid = 1;
  cudaMemsetAsync(kb->st.p, 0, sizeof(K6State), s);
  cudaMemsetAsync(kb->tk.p, 0, sizeof(uint32_t) * (nw_cap + dw_cap) * 2, s);
  cudaMemsetAsync(kb->cstat.p, 0, sizeof(unsigned long long) * nc, s);
  K6Args a;
  memset(&a, 0, sizeof(a));
  a.B = B;
  a.x_off = x_off;
  a.x_idx = x_idx;
  a.x_val = x_val;
  a.masks = masks;
  a.mask_stride = mask_stride;
  a.x_ids = x_ids && sem == kMinSelect2nd ? 1 : 0;
  a.y_off = y_off;
  a.y_cap = y_cap;
  a.y_idx = y_idx;
  a.y_val = y_val;
  a.d_nnz_y = d_nnz_y;
  a.colptr = A.colptr;
  a.rowidx = A.rowidx;
  a.nhot = h->ws.nhot;
  a.rowidx_t = h->ws.nhot > 0 ? h->ws.rowidx_k2 : A.rowidx;
  a.hot_rows = h->ws.hot_rows;
  a.val = A.val;
  a.jc = A.jc;
  a.aux = A.aux;
  a.aux_shift = A.aux_shift;
  a.m = A.m;
  a.n = A.n;
  a.nnz = A.nnz;
  a.lwb = lwb;
  a.nb = nb;
  a.q = q;
  a.win = win;
  a.nc = (int32_t)nc;
  a.tw = (int32_t)tw;
  a.nw_cap = (int32_t)nw_cap;
  a.tiles_cap = (int32_t)tiles;
  a.st = kb->st.p;
  a.tk = kb->tk.p;
  a.wt0 = kb->wt0.p;
  a.wl0 = kb->wl0.p;
  a.cstat = kb->cstat.p;
  a.xp = kb->xp.p;
  a.cp = kb->cp.p;
  a.fW = kb->fW.p;
  a.ffc = kb->ffc.p;
  a.ftb = kb->ftb.p;
  a.lb = kb->lb.p;
  a.sl = kb->sl.p;
  a.cw = kb->cw.p;
  a.cb = kb->cb.p;
  a.cx = kb->cx.p;
  a.tk0 = kb->tk0.p;
  a.tf = kb->tf.p;
  a.brow = kb->brow.p;
  a.bval = kb->bval.p;
  a.toff = kb->toff.p;
  a.bstat = kb->bstat.p;
  a.status = &h->ws.st->status;
  a.direct_min = direct ? std::max<int32_t>(K6_SMALL_MAX + 1, A.m / 2) : 0;
  a.dslots = dslots;
  a.dacc = direct ? kb->dacc.p : nullptr;
  a.dstat = kb->dstat.p;
  a.nrt = nrt;
  a.ld = kb->ld.p;
  a.fdi = kb->fdi.p;
  a.dwt0 = kb->dwt0.p;
  a.dw_cap = (int32_t)dw_cap;
  const size_t smem = k6_smem(lwb, nb);
  if (smem > SMEM_PER_BLOCK_MAX) return fail(SPMSPV_ERR_UNSUPPORTED, "batched layout too large");
  const bool q8 = q == K2_IMAX * K6_THREADS;
  switch (sem) {
    case kPlusTimes:
      e = q8 ? k6_launch<kPlusTimes, K2_IMAX>(kb, a, smem, h->sm_count, s)
             : k6_launch<kPlusTimes, K2_IMAX / 2>(kb, a, smem, h->sm_count, s);
      break;
    case kMinSelect2nd:
      e = q8 ? k6_launch<kMinSelect2nd, K2_IMAX>(kb, a, smem, h->sm_count, s)
             : k6_launch<kMinSelect2nd, K2_IMAX / 2>(kb, a, smem, h->sm_count, s);
      break;
    default:
      e = q8 ? k6_launch<kOrAnd, K2_IMAX>(kb, a, smem, h->sm_count, s)
             : k6_launch<kOrAnd, K2_IMAX / 2>(kb, a, smem, h->sm_count, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "batched persistent launch");
  h->last_stream = s;
  return SPMSPV_OK;
}

}  // namespace spmspv

using namespace spmspv;

extern "C" int spmspv_batched_phase_times(spmspv_handle* h, double* ms, int32_t capacity, int32_t* waves) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!ms || capacity < 0) return fail(SPMSPV_ERR_ARG, "bad arguments");
  const K6Buffers* kb = (const K6Buffers*)h->k6;
  if (!kb || !kb->st.p) return fail(SPMSPV_ERR_STATE, "no persistent batched launch on this handle yet");
  cudaError_t e = cudaStreamSynchronize(h->last_stream);
  K6State st;
  if (e == cudaSuccess) e = cudaMemcpy(&st, kb->st.p, sizeof(st), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "phase times");
  const unsigned long long* t = st.t;
  const unsigned long long end = t[K6_STAMPS - 1];
  auto at = [&](int k) { return k < K6_STAMPS - 1 && t[k] ? t[k] : end; };
  double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  v[0] = (double)(at(1) - t[0]) * 1e-6;
  v[1] = (double)(at(2) - at(1)) * 1e-6;
  v[2] = (double)(at(3) - at(2)) * 1e-6;
  // the direct waves (two barriers each), then the bucket waves
  const int ndw = st.n_dwaves;
  for (int dw = 0; dw < ndw; ++dw) {
    const int b0 = 3 + 2 * dw;
    v[6] += (double)(at(b0 + 1) - at(b0)) * 1e-6;
    v[7] += (double)(at(b0 + 2) - at(b0 + 1)) * 1e-6;
  }
  const int base = 3 + 2 * ndw;
  const int nw = st.n_waves;
  if (nw == 0) {
    v[3] = (double)(end - at(base)) * 1e-6;
  } else {
    for (int w = 0; w < nw; ++w) {
      const int b0 = base + 2 * w;
      v[3] += (double)(at(b0 + 1) - at(b0)) * 1e-6;
      v[4] += (double)((w + 1 < nw ? at(b0 + 2) : end) - at(b0 + 1)) * 1e-6;
    }
  }
  v[5] = (double)(end - t[0]) * 1e-6;
  for (int i = 0; i < 8 && i < capacity; ++i) ms[i] = v[i];
  if (waves) *waves = nw;
  return SPMSPV_OK;
}

