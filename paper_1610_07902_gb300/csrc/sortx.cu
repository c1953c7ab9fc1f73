// Presort of the input vector by index.  Sec. III-A (cache efficiency) notes
// that sorting x beforehand makes the column accesses of Step 1 more local
// when x is denser, since consecutive entries then touch nearby columns; the
// experiments of Sec. IV keep x and y sorted for that reason (Sec. IV-B).
//
// Indices are distinct and below n, so the sort is a counting sort over the
// index range: one kernel sets a bit per entry in an n-bit bitmap and parks
// the value in a dense array; a second kernel compacts the bitmap in order
// (256-word tiles taken from a ticket, block scan of the popcounts, decoupled
// look-back across tiles), writes (j, value) pairs ascending and clears the
// bitmap behind it for the next call.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "device_util.cuh"
#include "handle.cuh"
#include "spmspv_internal.cuh"

namespace spmspv {
namespace {

constexpr int SX_THREADS = 256;
constexpr int SX_WPT = 1;                              // bitmap words per thread
constexpr int SX_TILE_WORDS = SX_THREADS * SX_WPT;     // 256 words = 8192 ids

__global__ void k_sortx_scatter(const int32_t* __restrict__ x_idx, const uint32_t* __restrict__ x_val,
                                int32_t f, int32_t n, uint32_t* __restrict__ bits,
                                uint32_t* __restrict__ dense, unsigned long long* __restrict__ status,
                                int32_t ntiles, DevState* st) {
  if (blockIdx.x == 0)
    for (int t = threadIdx.x; t <= ntiles; t += blockDim.x) status[t] = 0ull;  // + the ticket word
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < f; k += gridDim.x * blockDim.x) {
    const int32_t j = x_idx[k];
    if ((uint32_t)j >= (uint32_t)n) {
      atomicOr(&st->status, ST_INDEX);
      continue;
    }
    atomicOr(&bits[j >> 5], 1u << (j & 31));
    if (x_val) dense[j] = x_val[k];
  }
}

__global__ void __launch_bounds__(SX_THREADS)
k_sortx_compact(uint32_t* __restrict__ bits, const uint32_t* __restrict__ dense, int32_t nw,
                int with_val, int32_t f, int32_t* __restrict__ out_idx, uint32_t* __restrict__ out_val,
                unsigned long long* status, int32_t ntiles, DevState* st) {
  __shared__ uint32_t s_tile;
  __shared__ int32_t s_scan[SX_THREADS / 32 + 1];
  __shared__ unsigned long long s_off;
  const int tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(reinterpret_cast<unsigned int*>(status + ntiles), 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const int64_t w0 = (int64_t)tile * SX_TILE_WORDS + (int64_t)tid * SX_WPT;
  uint32_t wv[SX_WPT];
  int32_t c = 0;
#pragma unroll
  for (int q = 0; q < SX_WPT; ++q) {
    wv[q] = w0 + q < nw ? bits[w0 + q] : 0u;
    c += __popc(wv[q]);
  }
  int32_t tot;
  const int32_t run = block_exclusive_sum<SX_THREADS>(c, s_scan, &tot);
  if (tid < 32) {
    const unsigned long long pre = warp_lookback(status, tile, (unsigned long long)tot, st);
    if (tid == 0) {
      s_off = pre;
      // repeated or out-of-range ids leave fewer sorted entries than nnz(x)
      if (tile == (uint32_t)ntiles - 1 && pre + (unsigned long long)tot != (unsigned long long)f)
        atomicOr(&st->status, ST_INDEX);
    }
  }
  __syncthreads();
  int64_t pos = (int64_t)s_off + run;
#pragma unroll
  for (int q = 0; q < SX_WPT; ++q) {
    uint32_t b = wv[q];
    if (!b) continue;
    bits[w0 + q] = 0u;
    while (b) {
      const int32_t j = (int32_t)((w0 + q) << 5) + __ffs(b) - 1;
      b &= b - 1u;
      out_idx[pos] = j;
      if (with_val) out_val[pos] = dense[j];
      ++pos;
    }
  }
}

}  // namespace

static int sortx_tiles(int32_t n) {
  const int32_t nw = (n + 31) / 32;
  return (nw + SX_TILE_WORDS - 1) / SX_TILE_WORDS;
}

int sort_x(spmspv_handle* h, const int32_t* x_idx, const uint32_t* x_val, int32_t f, cudaStream_t s) {
  const int32_t n = h->A.n;
  const int32_t nw = (n + 31) / 32;
  const int ntiles = sortx_tiles(n);
  if (!h->sx_bits) {
    cudaError_t e = cudaMalloc(&h->sx_bits, sizeof(uint32_t) * (size_t)nw);
    if (e == cudaSuccess) e = cudaMalloc(&h->sx_dense, sizeof(uint32_t) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&h->sx_idx, sizeof(int32_t) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&h->sx_val, sizeof(uint32_t) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&h->sx_status, sizeof(unsigned long long) * (size_t)(ntiles + 1));
    if (e == cudaSuccess) e = cudaMemset(h->sx_bits, 0, sizeof(uint32_t) * (size_t)nw);
    if (e != cudaSuccess) {
      release_sortx(h);
      cudaGetLastError();
      return fail(SPMSPV_ERR_OOM, "x presort buffers: %s", cudaGetErrorString(e));
    }
  }
  const int sgrid = std::max(1, std::min(h->sm_count * 8, (f + 255) / 256));
  k_sortx_scatter<<<sgrid, 256, 0, s>>>(x_idx, x_val, f, n, h->sx_bits, h->sx_dense, h->sx_status, ntiles,
                                        h->ws.st);
  k_sortx_compact<<<ntiles, SX_THREADS, 0, s>>>(h->sx_bits, h->sx_dense, nw, x_val ? 1 : 0, f, h->sx_idx,
                                                h->sx_val, h->sx_status, ntiles, h->ws.st);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SPMSPV_OK : cuda_fail(e, "x presort");
}

void release_sortx(spmspv_handle* h) {
  cudaFree(h->sx_bits);
  cudaFree(h->sx_dense);
  cudaFree(h->sx_idx);
  cudaFree(h->sx_val);
  cudaFree(h->sx_status);
  h->sx_bits = nullptr;
  h->sx_dense = nullptr;
  h->sx_idx = nullptr;
  h->sx_val = nullptr;
  h->sx_status = nullptr;
}

}  // namespace spmspv
