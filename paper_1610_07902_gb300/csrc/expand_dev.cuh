// Device helpers of the expand and merge steps shared by the single-call
// kernels (kernels.cu) and the persistent batched kernel (batched_k6.cu):
// the semirings' identities and shared-memory updates, and the gather of a
// warp's products from a merge-path tile.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "device_util.cuh"
#include "spmspv_internal.cuh"

namespace spmspv {

// ------------------------------------------------------------------------
// Semiring helpers
// ------------------------------------------------------------------------
template <int SEM>
__device__ __forceinline__ uint32_t sr_identity() {
  return SEM == kMinSelect2nd ? 0x7fffffffu : 0u;  // min: INT32_MAX; plus: +0.0f
}

// SPA update in shared memory (atomic: other threads may hit the same row)
template <int SEM>
__device__ __forceinline__ void spa_apply(uint32_t* spa, uint32_t r, uint32_t v) {
  if (SEM == kPlusTimes) atomicAdd(reinterpret_cast<float*>(spa + r), __uint_as_float(v));
  else if (SEM == kMinSelect2nd) atomicMin(reinterpret_cast<int*>(spa + r), (int)v);
}

// The value no merge produces (dense SPA form): -0.0f for (+,*), INT32_MAX
// for (min, select2nd) in BFS, where x values are vertex ids.
template <int SEM>
__device__ __forceinline__ uint32_t spa_empty() {
  return SEM == kPlusTimes ? 0x80000000u : 0x7fffffffu;
}

// The products of one warp's chunk: entry lookup, coalesced loads of row ids
// and values, the multiply (FULL: the tile holds items*K2_THREADS products,
// no bounds test).
template <int SEM, int IT, bool FULL>
__device__ __forceinline__ void k2_gather(const int32_t* __restrict__ rowidx, const float* __restrict__ val,
                                          const uint32_t* hbits, const int32_t* kbase, const uint32_t* kx,
                                          int items, int warp, int lane, int32_t p0, int32_t np, int64_t nnz,
                                          uint32_t (&rrow)[K2_IMAX], uint32_t (&rval)[K2_IMAX]) {
  const int w0 = warp * items;  // bitmap word of this warp's first 32 products
  const int32_t pw0 = w0 * 32 + lane;
  int ent = 0;                  // entry starts before word w0
  for (int j = lane; j < w0; j += 32) ent += __popc(hbits[j]);
  ent = __reduce_add_sync(0xffffffffu, ent);
  const uint32_t le = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
  uint32_t xi[K2_IMAX];
  float av[K2_IMAX];
  // every item's address, then all loads in flight at once
#pragma unroll
  for (int i = 0; i < K2_IMAX; ++i) {
    rrow[i] = 0xffffffffu;
    xi[i] = 0u;
    av[i] = 1.0f;
    if (IT ? i < IT : i < items) {
      const int32_t pl = pw0 + 32 * i;
      const uint32_t hw = hbits[w0 + i];
      const int e = ent + __popc(hw & le);
      ent += __popc(hw);
      if (FULL || pl < np) {
        const int32_t pos = kbase[e] + p0 + pl;
        xi[i] = kx[e];
        if ((uint32_t)pos < (uint32_t)nnz) {  // always true with valid inputs
          rrow[i] = (uint32_t)ld_stream(rowidx + pos);
          if (SEM == kPlusTimes && val) av[i] = ld_stream(val + pos);
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < K2_IMAX; ++i) {
    uint32_t v = 0u;
    if (SEM == kPlusTimes) {
      v = __float_as_uint(__fmul_rn(av[i], __uint_as_float(xi[i])));
      if (v == 0x80000000u) v = 0u;  // -0.0 -> +0.0: K3's dense SPA reserves -0.0 for "empty"
    } else if (SEM == kMinSelect2nd) {
      v = xi[i];
    }
    rval[i] = v;
  }
}

// The mask bit of every item's row (bit i of the result for item i; hub
// labels m + h read the bit of hrow[h]; items without a product read
// nothing), with every item's load issued before any result is used.
__device__ __forceinline__ uint32_t k2_mask_bits(const uint32_t* __restrict__ mask,
                                                 const uint32_t (&rrow)[K2_IMAX], uint32_t m, uint32_t nhot,
                                                 const int32_t* hrow) {
  uint32_t w[K2_IMAX], r[K2_IMAX];
#pragma unroll
  for (int i = 0; i < K2_IMAX; ++i) {
    r[i] = rrow[i];
    if (r[i] != 0xffffffffu && r[i] >= m) r[i] = r[i] - m < nhot ? (uint32_t)hrow[r[i] - m] : 0xffffffffu;
    w[i] = r[i] != 0xffffffffu ? __ldg(mask + (r[i] >> 5)) : 0u;
  }
  uint32_t bits = 0u;
#pragma unroll
  for (int i = 0; i < K2_IMAX; ++i) bits |= ((w[i] >> (r[i] & 31)) & 1u) << i;
  return bits;
}

}  // namespace spmspv
