// End-to-end form of the product (Algorithm 1 with x and y in host memory):
// x is copied to device buffers the handle keeps, the product runs as
// spmspv_run does, nnz(y) comes back first (one synchronisation of the
// stream) and then exactly that many entries of y.  The copies run on the
// copy engines: kernels reading x and writing y in page-locked host memory
// across the host link were no faster on this GPU (x read in place: the
// same time; a 12.8 MB y written in place by the merge kernel: about 50 us
// more than one copy after it).  The paper's
// product reads and writes host memory directly (a CPU method); on the GPU
// these copies are the price of the same interface.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "handle.cuh"
#include "spmspv.h"

namespace spmspv {

namespace {

struct HostIO {
  int32_t* x_idx = nullptr;
  uint32_t* x_val = nullptr;
  size_t x_cap = 0;
  int32_t* y_idx = nullptr;
  uint32_t* y_val = nullptr;
  size_t y_cap = 0;
  int32_t* d_nnz = nullptr;  // device nnz(y)
  int32_t* h_nnz = nullptr;  // page-locked copy of it
};

// A pair of device arrays of at least `need` 32-bit entries (contents are
// not kept when they grow).
cudaError_t grow_pair(int32_t** a, uint32_t** b, size_t* cap, size_t need) {
  if (need <= *cap && *a) return cudaSuccess;
  cudaFree(*a);
  cudaFree(*b);
  *a = nullptr;
  *b = nullptr;
  *cap = 0;
  const size_t n = std::max<size_t>(need, 1);
  cudaError_t e = cudaMalloc(a, sizeof(int32_t) * n);
  if (e == cudaSuccess) e = cudaMalloc(b, sizeof(uint32_t) * n);
  if (e == cudaSuccess) *cap = n;
  return e;
}

}  // namespace

void release_hostio(spmspv_handle* h) {
  HostIO* io = (HostIO*)h->hostio;
  if (!io) return;
  cudaFree(io->x_idx);
  cudaFree(io->x_val);
  cudaFree(io->y_idx);
  cudaFree(io->y_val);
  cudaFree(io->d_nnz);
  cudaFreeHost(io->h_nnz);
  delete io;
  h->hostio = nullptr;
}

}  // namespace spmspv

using namespace spmspv;

extern "C" int spmspv_run_host(spmspv_handle* h, int semiring, const int32_t* x_idx, const void* x_val,
                               int32_t nnz_x, const uint32_t* mask, uint32_t opts, int32_t* y_idx, void* y_val,
                               int32_t y_capacity, int32_t* nnz_y, spmspv_stream_t stream) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (semiring < 0 || semiring > 2) return fail(SPMSPV_ERR_ARG, "unknown semiring %d", semiring);
  if (nnz_x < 0 || nnz_x > h->A.n) return fail(SPMSPV_ERR_ARG, "nnz_x = %d outside [0, n]", nnz_x);
  if (nnz_x > 0 && !x_idx) return fail(SPMSPV_ERR_ARG, "x_idx is NULL");
  const bool values = semiring != SPMSPV_OR_AND_BOOL;
  if (nnz_x > 0 && values && !x_val) return fail(SPMSPV_ERR_ARG, "x_val is NULL");
  if (y_capacity < 0) return fail(SPMSPV_ERR_ARG, "y_capacity < 0");
  if (y_capacity > 0 && !y_idx) return fail(SPMSPV_ERR_ARG, "y_idx is NULL");
  if (y_capacity > 0 && values && !y_val) return fail(SPMSPV_ERR_ARG, "y_val is NULL");
  if (!nnz_y) return fail(SPMSPV_ERR_ARG, "nnz_y is NULL");
  if (nnz_x == 0) {  // an empty x gives an empty y (as in spmspv_run)
    h->last_stream = (cudaStream_t)stream;
    h->last_empty = 1;
    *nnz_y = 0;
    return SPMSPV_OK;
  }
  if (!h->hostio) h->hostio = new HostIO();
  HostIO* io = (HostIO*)h->hostio;
  cudaError_t e = grow_pair(&io->x_idx, &io->x_val, &io->x_cap, (size_t)nnz_x);
  if (e == cudaSuccess) e = grow_pair(&io->y_idx, &io->y_val, &io->y_cap, (size_t)y_capacity);
  if (e == cudaSuccess && !io->d_nnz) e = cudaMalloc(&io->d_nnz, sizeof(int32_t));
  if (e == cudaSuccess && !io->h_nnz) e = cudaMallocHost(&io->h_nnz, sizeof(int32_t));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(SPMSPV_ERR_OOM, "host-buffer staging: %s", cudaGetErrorString(e));
  }
  cudaStream_t s = (cudaStream_t)stream;
  e = cudaMemcpyAsync(io->x_idx, x_idx, sizeof(int32_t) * nnz_x, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && values)
    e = cudaMemcpyAsync(io->x_val, x_val, sizeof(uint32_t) * nnz_x, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "x to the device");
  rc = spmspv_run(h, semiring, io->x_idx, values ? (const void*)io->x_val : nullptr, nnz_x, mask, opts, io->y_idx,
                  values ? (void*)io->y_val : nullptr, y_capacity, io->d_nnz, stream);
  if (rc != SPMSPV_OK) {
    cudaStreamSynchronize(s);  // no copy may still read the caller's x
    return rc;
  }
  e = cudaMemcpyAsync(io->h_nnz, io->d_nnz, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "nnz(y) to the host");
  const int32_t k = *io->h_nnz;
  *nnz_y = k;
  const int32_t c = std::min(std::max(k, 0), y_capacity);
  if (c > 0) {
    e = cudaMemcpyAsync(y_idx, io->y_idx, sizeof(int32_t) * c, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && values)
      e = cudaMemcpyAsync(y_val, io->y_val, sizeof(uint32_t) * c, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "y to the host");
  }
  return SPMSPV_OK;
}
