// spmspv_run_noalloc: the SpMSpV path with its scratch in a fixed,
// library-owned device array instead of a handle's workspace.
//
// Some callers cannot call cudaMalloc: code that must not stall the device
// (cudaMalloc may synchronise it), code that runs inside a host process
// whose allocator owns all device memory, or code whose memory budget is
// fixed when it is loaded.  This entry point lets them run a product with
// inputs and outputs they already own; it allocates nothing.
//
// The scratch is one file-scope array of NA_SCRATCH_BYTES (about 7 MB) that
// every GPU loading the library holds until the process exits.  Every call
// shares it: two calls that overlap on the GPU (different streams, or
// different host threads without ordering) race on it and give undefined
// results.  Each call clears the part that must start at zero, so a call
// never depends on what the previous one left behind.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "handle.cuh"
#include "spmspv_internal.cuh"

namespace spmspv {
namespace {

constexpr int NA_MAX_X = 1 << 16;          // nnz(x)
constexpr int64_t NA_MAX_NNZ = 1 << 20;    // nnz(A)
constexpr int32_t NA_MAX_M = 1 << 22;      // rows of A
constexpr int NA_NB_MAX = 512;             // fine buckets for m <= NA_MAX_M
constexpr int NA_TILES = (int)(NA_MAX_NNZ / QF) + 2;
constexpr int NA_K1_TILES = NA_MAX_X / K1_TILE + 1;
constexpr int NA_MAX_DEVICES = 64;

constexpr size_t na_align(size_t v) { return (v + 255) / 256 * 256; }
// zeroed at every call: state, look-back words, fill counters, bucket counts
constexpr size_t NA_OFF_ST = 0;
constexpr size_t NA_OFF_K1S = NA_OFF_ST + na_align(sizeof(DevState));
constexpr size_t NA_OFF_BF = NA_OFF_K1S + na_align(sizeof(unsigned long long) * NA_K1_TILES);
constexpr size_t NA_OFF_K3S = NA_OFF_BF + na_align(sizeof(int32_t) * NA_NB_MAX * BFILL_STRIDE);
constexpr size_t NA_OFF_CNT = NA_OFF_K3S + na_align(sizeof(unsigned long long) * NA_NB_MAX);
constexpr size_t NA_ZERO_BYTES = NA_OFF_CNT + na_align(sizeof(int32_t) * (NA_NB_MAX + 4));
// written before they are read in every call
constexpr size_t NA_OFF_RB = NA_ZERO_BYTES;
constexpr size_t NA_OFF_CW = NA_OFF_RB + na_align(sizeof(int32_t) * (NA_NB_MAX + 1));
constexpr size_t NA_OFF_CB = NA_OFF_CW + na_align(sizeof(int32_t) * (NA_MAX_X + 1));
constexpr size_t NA_OFF_CX = NA_OFF_CB + na_align(sizeof(int32_t) * NA_MAX_X);
constexpr size_t NA_OFF_TK = NA_OFF_CX + na_align(sizeof(uint32_t) * NA_MAX_X);
constexpr size_t NA_OFF_BR = NA_OFF_TK + na_align(sizeof(int32_t) * NA_TILES);
constexpr size_t NA_OFF_BV = NA_OFF_BR + na_align(sizeof(uint16_t) * NA_MAX_NNZ);
constexpr size_t NA_SCRATCH_BYTES = NA_OFF_BV + na_align(sizeof(uint32_t) * NA_MAX_NNZ);

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_SCRATCH_BYTES];

namespace {

struct DeviceSetup {
  bool ready = false;
  unsigned char* scratch = nullptr;  // device address of g_noalloc_scratch
  int sm_count = 0;
  int k2_grid = 0;
};

std::mutex g_setup_mutex;
DeviceSetup g_setup[NA_MAX_DEVICES];

// Exclusive prefix of the per-bucket nonzero counts: the first slot of
// every bucket's region (one CTA; nb <= NA_NB_MAX).
__global__ void k_region_starts(const int32_t* __restrict__ counts, int nb, int32_t* __restrict__ rbase) {
  __shared__ int32_t s[NA_NB_MAX + 1];
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s[i] = counts[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t acc = 0;
    for (int i = 0; i < nb; ++i) {
      rbase[i] = acc;
      acc += s[i];
    }
    rbase[nb] = acc;
  }
}

// A matrix with row ids outside [0, m) (counted while sizing the bucket
// regions) or an x with out-of-range or repeated indices (flagged by the work
// scan) makes the result undefined: the kernels drop what they cannot place
// and this one-thread kernel then reports the call as failed with
// *d_nnz_y = -1.
__global__ void k_noalloc_report(const unsigned int* __restrict__ bad, const DevState* __restrict__ st,
                                 int32_t* __restrict__ d_nnz_y) {
  if (*bad != 0u || (st->status & ST_INDEX) != 0u) *d_nnz_y = -1;
}

int setup_device(int dev, DeviceSetup** out) {
  if (dev < 0 || dev >= NA_MAX_DEVICES)
    return fail(SPMSPV_ERR_UNSUPPORTED, "device %d is beyond the %d devices supported", dev,
                NA_MAX_DEVICES);
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup& d = g_setup[dev];
  if (!d.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    e = cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device attribute");
    e = set_kernel_attributes(k2_smem_bytes(NB_K2_MAX, true), k3_smem_bytes(LWB_MAX));
    if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
    d.k2_grid = d.sm_count * k2_blocks_per_sm(kPlusTimes, k2_smem_bytes(NA_NB_MAX, false));
    d.scratch = (unsigned char*)p;
    d.ready = true;
  }
  *out = &d;
  return SPMSPV_OK;
}

}  // namespace
}  // namespace spmspv

using namespace spmspv;

extern "C" int spmspv_run_noalloc(int32_t m, int32_t n, int64_t nnz, const int32_t* colptr,
                                  const int32_t* rowidx, const void* val, int val_type,
                                  int semiring, const int32_t* x_idx, const void* x_val,
                                  int32_t nnz_x, const uint32_t* mask, uint32_t opts,
                                  int32_t* y_idx, void* y_val, int32_t y_capacity,
                                  int32_t* d_nnz_y, spmspv_stream_t stream) {
  if (m < 1 || n < 1) return fail(SPMSPV_ERR_ARG, "m and n must be >= 1 (got %d, %d)", m, n);
  if (m > NA_MAX_M)
    return fail(SPMSPV_ERR_UNSUPPORTED, "no-alloc path: m = %d exceeds its maximum of %d rows", m,
                NA_MAX_M);
  if (nnz < 0) return fail(SPMSPV_ERR_ARG, "nnz < 0");
  if (nnz > NA_MAX_NNZ)
    return fail(SPMSPV_ERR_UNSUPPORTED,
                "no-alloc path: nnz(A) = %lld exceeds its maximum of %lld nonzeros",
                (long long)nnz, (long long)NA_MAX_NNZ);
  if (nnz_x < 0 || nnz_x > n) return fail(SPMSPV_ERR_ARG, "nnz_x = %d outside [0, n]", nnz_x);
  if (nnz_x > NA_MAX_X)
    return fail(SPMSPV_ERR_UNSUPPORTED, "no-alloc path: nnz(x) = %d exceeds its maximum of %d",
                nnz_x, NA_MAX_X);
  if (!colptr || (nnz > 0 && !rowidx)) return fail(SPMSPV_ERR_ARG, "colptr or rowidx is NULL");
  if (val_type != SPMSPV_VAL_NONE && val_type != SPMSPV_VAL_F32)
    return fail(SPMSPV_ERR_ARG, "unknown val_type %d", val_type);
  if (val_type == SPMSPV_VAL_F32 && nnz > 0 && !val) return fail(SPMSPV_ERR_ARG, "val is NULL");
  if (semiring < 0 || semiring > 2) return fail(SPMSPV_ERR_ARG, "unknown semiring %d", semiring);
  if (nnz_x > 0 && !x_idx) return fail(SPMSPV_ERR_ARG, "x_idx is NULL");
  if (nnz_x > 0 && semiring != SPMSPV_OR_AND_BOOL && !x_val) return fail(SPMSPV_ERR_ARG, "x_val is NULL");
  if (y_capacity < 0) return fail(SPMSPV_ERR_ARG, "y_capacity < 0");
  if (y_capacity > 0 && !y_idx) return fail(SPMSPV_ERR_ARG, "y_idx is NULL");
  if (y_capacity > 0 && semiring != SPMSPV_OR_AND_BOOL && !y_val) return fail(SPMSPV_ERR_ARG, "y_val is NULL");
  if (!d_nnz_y) return fail(SPMSPV_ERR_ARG, "d_nnz_y is NULL");
  if (opts & (SPMSPV_SCHED_FORCE | SPMSPV_SCHED_AUTO))
    return fail(SPMSPV_ERR_UNSUPPORTED, "no-alloc path runs the default schedule only");

  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  DeviceSetup* d = nullptr;
  int rc = setup_device(dev, &d);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;

  // bucket geometry, as a handle would choose it
  int lwb_hi = 0;
  while (((int64_t)1 << lwb_hi) < m) ++lwb_hi;
  lwb_hi -= 7;
  if (lwb_hi < LWB_MIN + 2) lwb_hi = LWB_MIN + 2;
  if (lwb_hi > LWB_MAX) lwb_hi = LWB_MAX;
  const int lwb_lo = lwb_hi - 2;
  const int nb_fine = (int)(((int64_t)m + (1 << lwb_lo) - 1) >> lwb_lo);

  unsigned char* base = d->scratch;
  Matrix A{};
  A.m = m;
  A.n = n;
  A.nnz = nnz;
  A.colptr = colptr;
  A.rowidx = rowidx;
  A.val = val_type == SPMSPV_VAL_F32 ? (const float*)val : nullptr;
  Workspace ws;
  ws.st = (DevState*)(base + NA_OFF_ST);
  ws.k1_status = (unsigned long long*)(base + NA_OFF_K1S);
  ws.bfill = (int32_t*)(base + NA_OFF_BF);
  ws.k3_status = (unsigned long long*)(base + NA_OFF_K3S);
  int32_t* counts = (int32_t*)(base + NA_OFF_CNT);
  ws.rbase = (int32_t*)(base + NA_OFF_RB);
  ws.cw = (int32_t*)(base + NA_OFF_CW);
  ws.cb = (int32_t*)(base + NA_OFF_CB);
  ws.cx = (uint32_t*)(base + NA_OFF_CX);
  ws.tile_k0 = (int32_t*)(base + NA_OFF_TK);
  ws.brow = (uint16_t*)(base + NA_OFF_BR);
  ws.bval = (uint32_t*)(base + NA_OFF_BV);
  ws.nhot = 0;
  ws.hot_rows = nullptr;
  ws.rowidx_k2 = nullptr;
  ws.pull_status = nullptr;
  ws.job = nullptr;
  ws.hot_start = nullptr;
  ws.hot_val = nullptr;
  ws.hot_touch = nullptr;
  ws.ydense = nullptr;  // no dense accumulator: every product runs the bucketed form

  e = cudaMemsetAsync(base, 0, NA_ZERO_BYTES, s);
  if (e != cudaSuccess) return cuda_fail(e, "clear no-alloc scratch");
  if (nnz_x == 0) {
    e = cudaMemsetAsync(d_nnz_y, 0, sizeof(int32_t), s);
    return e == cudaSuccess ? SPMSPV_OK : cuda_fail(e, "memset nnz_y");
  }
  // bucket regions of this matrix: nonzeros per row range, prefix-summed
  if (nnz > 0) {
    e = launch_bucket_sizes(A, lwb_lo, nb_fine, counts, (unsigned int*)(counts + NA_NB_MAX), s);
    if (e != cudaSuccess) return cuda_fail(e, "bucket size launch");
  }
  k_region_starts<<<1, 256, 0, s>>>(counts, nb_fine, ws.rbase);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "region start launch");

  Sched sc;
  sc.id = 5;  // the default schedule: 4096-product tiles, widest buckets
  sc.dir = 0;
  sc.q = 2 * QF;
  sc.lwb = lwb_lo + 2;
  const int k1_grid = (int)((nnz_x + K1_TILE - 1) / K1_TILE);
  e = launch_k1(semiring, A, ws, nb_fine, x_idx, (const uint32_t*)x_val, nnz_x, nullptr, k1_grid,
                &sc, s);
  if (e != cudaSuccess) return cuda_fail(e, "work scan launch");
  e = launch_k2(semiring, A, ws, lwb_lo, nb_fine, mask, (opts & SPMSPV_MASK_COMPLEMENT) ? 1 : 0,
                d->k2_grid, k2_smem_bytes(nb_fine, false), s, 0, sc.q);
  if (e != cudaSuccess) return cuda_fail(e, "expand/scatter launch");
  const int nb = (int)(((int64_t)m + (1 << sc.lwb) - 1) >> sc.lwb);
  const size_t k3_smem = k3_smem_bytes(sc.lwb);
  const int k3_grid = std::max(1, std::min(nb, d->sm_count * k3_blocks_per_sm(semiring, k3_smem)));
  e = launch_k3(semiring, false, A, ws, lwb_lo, nb_fine, y_idx, (uint32_t*)y_val, y_capacity,
                d_nnz_y, nullptr, k3_grid, k3_smem, s);
  if (e != cudaSuccess) return cuda_fail(e, "bucket merge launch");
  k_noalloc_report<<<1, 1, 0, s>>>((const unsigned int*)(counts + NA_NB_MAX), ws.st, d_nnz_y);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "index report launch");
  return SPMSPV_OK;
}
