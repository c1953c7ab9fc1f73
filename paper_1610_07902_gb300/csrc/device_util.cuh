// Device helpers shared by the kernel translation units (inlined in each).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "spmspv_internal.cuh"

namespace spmspv {

// ------------------------------------------------------------------------
// small device helpers
// ------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long lb_load(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void lb_store(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add_u32(uint32_t* p, uint32_t v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid barrier of a kernel whose CTAs are all resident (cooperative launch).
// `count` only grows during the launch (zero when it starts): barrier number
// `epoch` (1, 2, ...) is passed once it reaches epoch * gridDim.x.  A CTA's
// arrival is a release add after its writes; the wait polls with acquire
// loads, at most SPIN_LIMIT times, after which it sets ST_TIMEOUT in
// *status and returns false (every CTA then leaves the kernel).
__device__ __forceinline__ bool grid_barrier(uint32_t* count, uint32_t epoch, uint32_t* status, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    red_release_add_u32(count, 1u);
    const uint32_t target = epoch * gridDim.x;
    int ok = 1;
    uint32_t spins = 0;
    while ((int32_t)(ld_acquire_u32(count) - target) < 0) {
      if (++spins > SPIN_LIMIT) {
        atomicOr(status, ST_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(20);
    }
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may be scheduled before the kernel ahead of it on the stream
// has finished; pdl_wait() returns once that kernel has completed and its
// writes are visible (a no-op after a plain launch), pdl_launch_next() lets
// the next such kernel be scheduled (a no-op when there is none).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Streaming load (evict-first): matrix entries are read once per call.
__device__ __forceinline__ int32_t ld_stream(const int32_t* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }

// Exclusive look-back prefix for tile `tile`, computed by one full warp:
// the warp publishes the tile's aggregate, then reads the status words of
// its LB_WIN*32 nearest predecessors at once and sums back to the nearest
// one that holds an inclusive prefix, sliding the window when none does.
// Waits are bounded: on give-up *err gets ST_TIMEOUT and the words still
// missing count as empty inclusive prefixes.
constexpr int LB_WIN = 4;

__device__ __forceinline__ unsigned long long warp_lookback(unsigned long long* status, uint32_t tile,
                                            unsigned long long agg, uint32_t* err,
                                            uint32_t spin_limit = SPIN_LIMIT) {
  const int lane = threadIdx.x & 31;
  if (tile == 0) {
    if (lane == 0) lb_store(status, LB_FLAG_INC | agg);
    return 0ull;
  }
  if (lane == 0) lb_store(status + tile, LB_FLAG_AGG | agg);
  unsigned long long excl = 0;
  int64_t base = (int64_t)tile - 1;
  for (;;) {
    // word k*32+lane of the window is predecessor base - (k*32 + lane)
    unsigned long long s[LB_WIN];
#pragma unroll
    for (int k = 0; k < LB_WIN; ++k) {
      const int64_t idx = base - (k * 32 + lane);
      s[k] = idx >= 0 ? lb_load(status + idx) : LB_FLAG_INC;
    }
    int first = -1;  // distance of the nearest inclusive prefix in the window
    uint32_t spins = 0;
    for (;;) {
      first = -1;
      bool all_ready = true;
#pragma unroll
      for (int k = 0; k < LB_WIN; ++k) {
        const unsigned im = __ballot_sync(0xffffffffu, (s[k] & LB_FLAG_MASK) == LB_FLAG_INC);
        const unsigned rm = __ballot_sync(0xffffffffu, (s[k] & LB_FLAG_MASK) != 0ull);
        if (first < 0) {
          if (im) {
            const int f0 = __ffs(im) - 1;
            const unsigned need = f0 == 31 ? 0xffffffffu : ((2u << f0) - 1u);
            if ((rm & need) != need) all_ready = false;
            first = k * 32 + f0;
          } else if (rm != 0xffffffffu) {
            all_ready = false;
          }
        }
      }
      if (all_ready) break;
      if (++spins > spin_limit) {
        if (lane == 0) atomicOr(err, ST_TIMEOUT);
#pragma unroll
        for (int k = 0; k < LB_WIN; ++k)
          if ((s[k] & LB_FLAG_MASK) == 0ull) s[k] = LB_FLAG_INC;
        continue;  // recompute `first` with the missing words as empty prefixes
      }
      __nanosleep(32);
#pragma unroll
      for (int k = 0; k < LB_WIN; ++k) {
        const int64_t idx = base - (k * 32 + lane);
        if ((s[k] & LB_FLAG_MASK) == 0ull && idx >= 0) s[k] = lb_load(status + idx);
      }
    }
    const int stop = first < 0 ? LB_WIN * 32 - 1 : first;
    unsigned long long v = 0;
#pragma unroll
    for (int k = 0; k < LB_WIN; ++k)
      if (k * 32 + lane <= stop) v += s[k] & LB_VAL_MASK;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    excl += v;
    if (first >= 0) break;
    base -= LB_WIN * 32;
  }
  if (lane == 0) lb_store(status + tile, LB_FLAG_INC | (excl + agg));
  return excl;
}

// The same, recording a timeout in the device state's status word.
__device__ __forceinline__ unsigned long long warp_lookback(unsigned long long* status, uint32_t tile,
                                            unsigned long long agg, DevState* st,
                                            uint32_t spin_limit = SPIN_LIMIT) {
  return warp_lookback(status, tile, agg, &st->status, spin_limit);
}

// Exclusive prefix sum over the block.  `sh` holds NT/32 + 1 shared
// entries; every thread receives the block total in *total.
template <int NT, typename T>
__device__ __forceinline__ T block_exclusive_sum(T v, T* sh, T* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    T w = lane < NT / 32 ? sh[lane] : T(0);
    T wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < NT / 32) sh[lane] = wi - w;
    if (lane == NT / 32 - 1) sh[NT / 32] = wi;
  }
  __syncthreads();
  const T r = sh[wid] + x - v;
  *total = sh[NT / 32];
  __syncthreads();
  return r;
}

// Appends the lanes of a warp whose `take` is set at counter[0]++, one atomic
// per warp; returns this lane's slot (meaningful where take is set).  Every
// lane of the warp must call it.
__device__ __forceinline__ int32_t warp_append(bool take, int32_t* counter) {
  const int lane = threadIdx.x & 31;
  const unsigned b = __ballot_sync(0xffffffffu, take);
  int32_t base = 0;
  if (lane == 0 && b) base = atomicAdd(counter, __popc(b));
  base = __shfl_sync(0xffffffffu, base, 0);
  return base + __popc(b & ((1u << lane) - 1u));
}

}  // namespace spmspv
