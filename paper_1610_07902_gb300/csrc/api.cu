// C ABI of the SpMSpV library (include/spmspv.h): handle life cycle,
// argument checks, schedule choice and the launch sequence of one product.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include <string>
#include <vector>

#include "handle.cuh"
#include "spmspv_internal.cuh"

using namespace spmspv;

namespace {
thread_local std::string g_last_error;
}

namespace spmspv {

// One profiled call: events[0] before the first stage, events[i+1] after
// stage stages[i].
struct ProfileCall {
  std::vector<cudaEvent_t> events;
  std::vector<int> stages;
};
using ProfileLog = std::vector<ProfileCall>;

void prof_call_begin(spmspv_handle* h, cudaStream_t s) {
  if (!h->prof) return;
  ProfileLog* log = (ProfileLog*)h->prof;
  log->emplace_back();
  cudaEvent_t e;
  cudaEventCreate(&e);
  cudaEventRecord(e, s);
  log->back().events.push_back(e);
}

void prof_mark(spmspv_handle* h, int stage, cudaStream_t s) {
  if (!h->prof) return;
  ProfileLog* log = (ProfileLog*)h->prof;
  if (log->empty()) return;
  cudaEvent_t e;
  cudaEventCreate(&e);
  cudaEventRecord(e, s);
  log->back().events.push_back(e);
  log->back().stages.push_back(stage);
}

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(SPMSPV_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

static int ilog2_ceil(int64_t v) {
  int l = 0;
  while (((int64_t)1 << l) < v) ++l;
  return l;
}

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int select_hot_rows(spmspv_handle* h);

// Work-scan CTAs needed to count the mask's bits in one pass of 4 words per thread.
static int mask_pass_grid(const spmspv_handle* h) {
  const int64_t words = ((int64_t)h->A.m + 31) / 32;
  return (int)std::min<int64_t>(h->k1_grid_max, (words + K1_THREADS * 4 - 1) / (K1_THREADS * 4));
}

Sched decode_schedule(const spmspv_handle* h, int id) {
  Sched s;
  s.id = id;
  s.dir = id / 6;
  s.q = ((id / 3) % 2) ? 2 * QF : QF;
  s.lwb = h->lwb_lo + id % 3;
  return s;
}

int check_handle(const spmspv_handle* h) {
  if (!h || h->magic != kHandleMagic) return fail(SPMSPV_ERR_STATE, "invalid or destroyed handle");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != h->device)
    return fail(SPMSPV_ERR_STATE, "handle belongs to device %d but device %d is current", h->device,
                dev);
  return SPMSPV_OK;
}

// Products from which a (+,*) call runs the direct form (0: never).
static int32_t plus_direct_min(const spmspv_handle* h) {
  if (!h->plus_direct || !h->ws.ydense) return 0;
  return (int32_t)std::min<int64_t>(INT32_MAX, (int64_t)h->A.m * PLUS_DIRECT_PER_ROW);
}

// K3 CTAs for the direct form's compaction: one per 8192-row tile, at most
// two per SM.
static int direct_k3_grid(const spmspv_handle* h) {
  const int64_t tiles = ((int64_t)h->A.m + 8191) / 8192;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, 2 * h->sm_count));
}

// The push-direction product: K1 -> K2 -> K3 on `s`.
int run_push(spmspv_handle* h, int sem, const int32_t* x_idx, const uint32_t* x_val, int f,
             const int32_t* f_dev, const uint32_t* mask, int mask_comp, const Sched& sc,
             int32_t* y_idx, uint32_t* y_val, int32_t y_cap, int32_t* d_nnz_y, bool bfs,
             uint32_t* mask_update, cudaStream_t s) {
  int k1_grid = f_dev ? h->k1_grid_dev
                      : (int)std::min<int64_t>(h->k1_grid_max, ((int64_t)f + K1_TILE - 1) / K1_TILE);
  if (h->k1_mask) k1_grid = std::max(k1_grid, mask_pass_grid(h));
  if (k1_grid < 1) k1_grid = 1;
  cudaError_t e;
  prof_call_begin(h, s);
  if (bfs) {
    e = launch_k1_bfs(h->A, h->ws, h->nb_fine, x_idx, f_dev, k1_grid, &sc, s, mask);
  } else {
    e = launch_k1(sem, h->A, h->ws, h->nb_fine, x_idx, x_val, f, f_dev, k1_grid, &sc, s,
                  h->k1_mask);
  }
  if (e != cudaSuccess) return cuda_fail(e, "work scan launch");
  prof_mark(h, SPMSPV_STAGE_SCAN, s);
  const int32_t pdm = bfs ? 0 : plus_direct_min(h);
  e = launch_k2(sem, h->A, h->ws, h->lwb_lo, h->nb_fine, mask, mask_comp, h->k2_grid, h->k2_smem, s, 0,
                sc.q, 0, pdm);
  if (e != cudaSuccess) return cuda_fail(e, "expand/scatter launch");
  prof_mark(h, SPMSPV_STAGE_SCATTER, s);
  const size_t k3_smem = k3_smem_bytes(sc.lwb);
  const int nb = (int)(((int64_t)h->A.m + (1 << sc.lwb) - 1) >> sc.lwb);
  int k3_grid = std::max(1, std::min(nb, h->sm_count * h->k3_bps[sc.lwb - h->lwb_lo]));
  if (pdm > 0) k3_grid = std::max(k3_grid, direct_k3_grid(h));
  e = launch_k3(sem, bfs, h->A, h->ws, h->lwb_lo, h->nb_fine, y_idx, y_val, y_cap, d_nnz_y,
                mask_update, k3_grid, k3_smem, s, 0, 0, 0, 0, pdm);
  if (e != cudaSuccess) return cuda_fail(e, "bucket merge launch");
  prof_mark(h, SPMSPV_STAGE_MERGE, s);
  return SPMSPV_OK;
}

int select_hot_rows(spmspv_handle* h) {
  const int32_t m = h->A.m;
  int32_t* d_deg = nullptr;
  cudaError_t e = cudaMalloc(&d_deg, sizeof(int32_t) * ((size_t)m + 1));
  if (e != cudaSuccess) return fail(SPMSPV_ERR_OOM, "row degree scratch: %s", cudaGetErrorString(e));
  int32_t* d_max = d_deg + m;
  cudaMemset(d_deg, 0, sizeof(int32_t) * ((size_t)m + 1));
  e = launch_row_degrees(h->A, d_deg, d_max, 0);
  int32_t maxdeg = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&maxdeg, d_max, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    cudaFree(d_deg);
    return cuda_fail(e, "row degrees");
  }
  if (maxdeg < HOT_MIN_DEG) {
    cudaFree(d_deg);
    h->ws.nhot = 0;
    return SPMSPV_OK;
  }
  std::vector<int32_t> deg((size_t)m);
  e = cudaMemcpy(deg.data(), d_deg, sizeof(int32_t) * (size_t)m, cudaMemcpyDeviceToHost);
  cudaFree(d_deg);
  if (e != cudaSuccess) return cuda_fail(e, "row degree copy");
  std::vector<int32_t> cand;
  for (int32_t i = 0; i < m; ++i)
    if (deg[i] >= HOT_MIN_DEG) cand.push_back(i);
  if ((int)cand.size() > HOT_MAX) {
    std::nth_element(cand.begin(), cand.begin() + HOT_MAX, cand.end(), [&](int32_t a, int32_t b) {
      return deg[a] != deg[b] ? deg[a] > deg[b] : a < b;
    });
    cand.resize(HOT_MAX);
  }
  std::sort(cand.begin(), cand.end());
  const int nh = (int)cand.size();
  std::vector<int32_t> rows(HOT_MAX, -1), start((size_t)h->nb_fine + 1, 0);
  std::vector<int32_t> hub_of_row((size_t)m, -1);
  for (int i = 0; i < nh; ++i) {
    rows[i] = cand[i];
    hub_of_row[cand[i]] = i;
    start[(cand[i] >> h->lwb_lo) + 1]++;
  }
  for (int i = 0; i < h->nb_fine; ++i) start[i + 1] += start[i];
  e = cudaMemcpy((void*)h->ws.hot_rows, rows.data(), sizeof(int32_t) * HOT_MAX, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy((void*)h->ws.hot_start, start.data(), sizeof(int32_t) * start.size(),
                   cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "hub row tables");
  // the row-id copy K2 reads: hub row r becomes m + its hub index
  int32_t* d_map = nullptr;
  e = cudaMalloc(&d_map, sizeof(int32_t) * (size_t)m);
  if (e != cudaSuccess) return fail(SPMSPV_ERR_OOM, "hub map scratch: %s", cudaGetErrorString(e));
  e = cudaMalloc(&h->rowidx_k2, sizeof(int32_t) * (size_t)(h->A.nnz > 0 ? h->A.nnz : 1));
  if (e != cudaSuccess) {
    cudaFree(d_map);
    h->rowidx_k2 = nullptr;
    return fail(SPMSPV_ERR_OOM, "hub row-id copy: %s", cudaGetErrorString(e));
  }
  e = cudaMemcpy(d_map, hub_of_row.data(), sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_relabel_hubs(h->A, d_map, h->rowidx_k2, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(d_map);
  if (e != cudaSuccess) return cuda_fail(e, "hub relabel");
  h->ws.rowidx_k2 = h->rowidx_k2;
  h->ws.nhot = nh;
  return SPMSPV_OK;
}

cudaError_t launch_pull(const spmspv_handle* h, int sem, bool bfs, const int32_t* x_idx,
                        const uint32_t* x_val, int f, const int32_t* f_dev, const uint32_t* mask,
                        int mask_comp, int early_exit, int32_t* y_idx, uint32_t* y_val,
                        int32_t y_cap, int32_t* d_nnz_y, uint32_t* visited, int only_pull,
                        cudaStream_t s);
int pull_available(const spmspv_handle* h, int sem);

// Learned schedule: work scan -> selector (on the device) -> the push kernels
// and, when the pull form is available, the pull kernels; each set runs only
// if the selector chose its direction.
int run_auto(spmspv_handle* h, int sem, const int32_t* x_idx, const uint32_t* x_val, int f,
             const uint32_t* mask, int mask_comp, int32_t* y_idx, uint32_t* y_val, int32_t y_cap,
             int32_t* d_nnz_y, cudaStream_t s, int early_exit) {
  // the selector is trained on masked, BFS-like calls; without a mask a pull
  // reads every row of A (an R-MAT hub row of 10^5 entries in one thread), so
  // an unmasked call stays push
  const int can_pull = mask ? pull_available(h, sem) : 0;
  int k1_grid = (int)std::max<int64_t>(1, std::min<int64_t>(h->k1_grid_max, ((int64_t)f + K1_TILE - 1) / K1_TILE));
  if (mask) k1_grid = std::max(k1_grid, mask_pass_grid(h));
  prof_call_begin(h, s);
  // the work scan's last CTA runs the selector (no launch of its own)
  SelArgs sa{};
  sa.w = h->sel_w;
  sa.allow_pull = can_pull;
  sa.lwb_lo = h->lwb_lo;
  cudaError_t e = launch_k1(sem, h->A, h->ws, h->nb_fine, x_idx, x_val, f, nullptr, k1_grid, nullptr, s,
                            mask, &sa);
  if (e != cudaSuccess) return cuda_fail(e, "work scan launch");
  prof_mark(h, SPMSPV_STAGE_SCAN, s);
  prof_mark(h, SPMSPV_STAGE_SELECT, s);
  const int32_t pdm = plus_direct_min(h);
  e = launch_k2(sem, h->A, h->ws, h->lwb_lo, h->nb_fine, mask, mask_comp, h->k2_grid, h->k2_smem, s,
                can_pull, 0, 0, pdm);
  if (e != cudaSuccess) return cuda_fail(e, "expand/scatter launch");
  prof_mark(h, SPMSPV_STAGE_SCATTER, s);
  const int lwb = h->lwb_lo + 2;  // shared memory for the widest bucket
  const int nb_max = (int)(((int64_t)h->A.m + (1 << h->lwb_lo) - 1) >> h->lwb_lo);
  int k3_grid = std::max(1, std::min(nb_max, h->sm_count * h->k3_bps[2]));
  if (pdm > 0) k3_grid = std::max(k3_grid, direct_k3_grid(h));
  e = launch_k3(sem, false, h->A, h->ws, h->lwb_lo, h->nb_fine, y_idx, y_val, y_cap, d_nnz_y,
                nullptr, k3_grid, k3_smem_bytes(lwb), s, can_pull, 0, 0, 0, pdm);
  if (e != cudaSuccess) return cuda_fail(e, "bucket merge launch");
  prof_mark(h, SPMSPV_STAGE_MERGE, s);
  if (can_pull) {
    e = launch_pull(h, sem, false, x_idx, x_val, f, nullptr, mask, mask_comp, early_exit, y_idx, y_val, y_cap,
                    d_nnz_y, nullptr, 1, s);
    if (e != cudaSuccess) return cuda_fail(e, "pull launch");
    prof_mark(h, SPMSPV_STAGE_PULL, s);
  }
  return SPMSPV_OK;
}

}  // namespace spmspv

extern "C" {

const char* spmspv_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace spmspv {

// DCSC set-up (Sec. II-C): checks the stored column ids and pointers and
// builds the auxiliary column index on the host, O(nzc + n / 2^aux_shift),
// then copies it to the device.
// The DCSC checks and auxiliary index on host arrays (no CUDA calls): jc
// strictly ascending in [0, n), cp from 0 to nnz and non-decreasing; then
// chunks of 2^s column ids, about as many as stored columns, and aux[k] = the
// first position whose id is at least k * 2^s, for k in [0, (n-1)/2^s + 1].
static int dcsc_index_host(int32_t n, int64_t nnz, int32_t nzc, const int32_t* jc, const int32_t* cp,
                           std::vector<int32_t>& aux, int& shift) {
  for (int32_t p = 0; p < nzc; ++p) {
    if (jc[p] < 0 || jc[p] >= n) return fail(SPMSPV_ERR_ARG, "jc[%d] = %d outside [0, n)", p, jc[p]);
    if (p > 0 && jc[p] <= jc[p - 1]) return fail(SPMSPV_ERR_ARG, "jc is not strictly ascending at %d", p);
    if (cp && cp[p + 1] < cp[p]) return fail(SPMSPV_ERR_ARG, "cp decreases at %d", p);
  }
  if (cp && (cp[0] != 0 || (int64_t)cp[nzc] != nnz)) return fail(SPMSPV_ERR_ARG, "cp must run from 0 to nnz");
  int s = 0;
  while (((int64_t)n >> s) > (int64_t)(nzc > 0 ? nzc : 1)) ++s;
  const int64_t naux = (((int64_t)n - 1) >> s) + 2;
  aux.assign((size_t)naux, 0);
  int32_t p = 0;
  for (int64_t k = 0; k < naux; ++k) {
    const int64_t first = k << s;
    while (p < nzc && (int64_t)jc[p] < first) ++p;
    aux[(size_t)k] = p;
  }
  shift = s;
  return SPMSPV_OK;
}

static int build_dcsc_index(spmspv_handle* h, int32_t n, int64_t nnz, int32_t nzc, const int32_t* jc,
                            const int32_t* cp) {
  std::vector<int32_t> hjc((size_t)nzc), hcp((size_t)nzc + 1);
  cudaError_t e = cudaMemcpy(hjc.data(), jc, sizeof(int32_t) * (size_t)nzc, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(hcp.data(), cp, sizeof(int32_t) * ((size_t)nzc + 1), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "DCSC arrays copy");
  std::vector<int32_t> haux;
  int s = 0;
  int rc = dcsc_index_host(n, nnz, nzc, hjc.data(), hcp.data(), haux, s);
  if (rc != SPMSPV_OK) return rc;
  const size_t naux = haux.size();
  if ((e = cudaMalloc(&h->dcsc_aux, sizeof(int32_t) * (size_t)naux)) != cudaSuccess)
    return fail(SPMSPV_ERR_OOM, "DCSC index: %s", cudaGetErrorString(e));
  if ((e = cudaMemcpy(h->dcsc_aux, haux.data(), sizeof(int32_t) * (size_t)naux, cudaMemcpyHostToDevice)) !=
      cudaSuccess)
    return cuda_fail(e, "DCSC index copy");
  h->A.jc = jc;
  h->A.aux = h->dcsc_aux;
  h->A.nzc = nzc;
  h->A.aux_shift = s;
  return SPMSPV_OK;
}

// Handle creation for CSC (jc == NULL) and DCSC (jc, nzc; colptr = the
// pointers of the stored columns).
static int create_impl(spmspv_handle** out, int32_t m, int32_t n, int64_t nnz, const int32_t* colptr,
                       const int32_t* rowidx, const void* val, int val_type, uint32_t flags,
                       const int32_t* jc, int32_t nzc) {
  if (!out) return fail(SPMSPV_ERR_ARG, "h is NULL");
  *out = nullptr;
  if (m < 1 || n < 1) return fail(SPMSPV_ERR_ARG, "m and n must be >= 1 (got %d, %d)", m, n);
  if (m > (1 << 26))
    return fail(SPMSPV_ERR_UNSUPPORTED, "m = %d exceeds 2^26 rows (bucket row width limit)", m);
  if (nnz < 0 || nnz >= ((int64_t)1 << 31)) return fail(SPMSPV_ERR_ARG, "nnz must be in [0, 2^31)");
  if (!colptr) return fail(SPMSPV_ERR_ARG, "colptr is NULL");
  if (nnz > 0 && !rowidx) return fail(SPMSPV_ERR_ARG, "rowidx is NULL");
  if (val_type != SPMSPV_VAL_NONE && val_type != SPMSPV_VAL_F32)
    return fail(SPMSPV_ERR_ARG, "unknown val_type %d", val_type);
  if (val_type == SPMSPV_VAL_F32 && nnz > 0 && !val)
    return fail(SPMSPV_ERR_ARG, "val is NULL for SPMSPV_VAL_F32");

  spmspv_handle* h = new spmspv_handle();  // value-initialised: every field zero or its default
  h->magic = kHandleMagic;
  cudaGetDevice(&h->device);
  cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
  h->A.m = m;
  h->A.n = n;
  h->A.nnz = nnz;
  h->A.colptr = colptr;
  h->A.rowidx = rowidx;
  h->A.val = val_type == SPMSPV_VAL_F32 ? (const float*)val : nullptr;
  h->flags = flags;
  if (jc) {
    int rc0 = build_dcsc_index(h, n, nnz, nzc, jc, colptr);
    if (rc0 != SPMSPV_OK) {
      cudaFree(h->dcsc_aux);
      delete h;
      return rc0;
    }
  }

  // bucket row widths: the widest gives about 128 buckets, the schedule
  // chooses among three widths
  int lwb_hi = ilog2_ceil(m) - 7;
  if (lwb_hi < LWB_MIN + 2) lwb_hi = LWB_MIN + 2;
  if (lwb_hi > LWB_MAX) lwb_hi = LWB_MAX;
  h->lwb_lo = lwb_hi - 2;
  h->nb_fine = (int)(((int64_t)m + (1 << h->lwb_lo) - 1) >> h->lwb_lo);
  if (h->nb_fine > NB_K2_MAX) {
    const int nb_fine = h->nb_fine;
    cudaFree(h->dcsc_aux);
    delete h;
    return fail(SPMSPV_ERR_UNSUPPORTED, "too many row-range buckets (%d)", nb_fine);
  }

  // workspace: one allocation, carved in 256-byte aligned pieces
  const int64_t ntile_fine = nnz / QF + 2;
  const int64_t nt1 = ((int64_t)n + K1_TILE - 1) / K1_TILE + 1;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  size_t o_st = take(sizeof(DevState));
  const size_t ncomp = (size_t)compaction_capacity(h->A);  // x entries with a non-empty column
  size_t o_cw = take(sizeof(int32_t) * (ncomp + 1));
  size_t o_cb = take(sizeof(int32_t) * ncomp);
  size_t o_cx = take(sizeof(uint32_t) * ncomp);
  size_t o_tk = take(sizeof(int32_t) * (size_t)ntile_fine);
  size_t o_k1s = take(sizeof(unsigned long long) * (size_t)nt1);
  size_t o_bf = take(sizeof(int32_t) * (size_t)h->nb_fine * BFILL_STRIDE);
  size_t o_k3s = take(sizeof(unsigned long long) * (size_t)h->nb_fine);
  size_t o_rb = take(sizeof(int32_t) * ((size_t)h->nb_fine + 1));
  size_t o_hr = take(sizeof(int32_t) * HOT_MAX);
  size_t o_hs = take(sizeof(int32_t) * ((size_t)h->nb_fine + 1));
  size_t o_hv = take(sizeof(uint32_t) * HOT_MAX);
  size_t o_ht = take(sizeof(uint32_t) * HOT_MAX);
  // bucket payload, padded to whole 8-entry chunks (K3 reads it 16 bytes at a time)
  const size_t nbe = (size_t)((nnz > 0 ? nnz : 1) + 7) / 8 * 8;
  size_t o_br = take(sizeof(uint16_t) * nbe);
  size_t o_bv = take(sizeof(uint32_t) * nbe);
  const size_t zero_bytes = o_br;  // everything before the bucket payload starts zeroed
  h->ws_bytes = off;
  cudaError_t e = cudaMalloc(&h->ws_base, h->ws_bytes);
  if (e != cudaSuccess) {
    cudaFree(h->dcsc_aux);
    delete h;
    cudaGetLastError();
    return fail(SPMSPV_ERR_OOM, "workspace of %zu bytes: %s", off, cudaGetErrorString(e));
  }
  char* b = (char*)h->ws_base;
  h->ws.st = (DevState*)(b + o_st);
  h->ws.cw = (int32_t*)(b + o_cw);
  h->ws.cb = (int32_t*)(b + o_cb);
  h->ws.cx = (uint32_t*)(b + o_cx);
  h->ws.tile_k0 = (int32_t*)(b + o_tk);
  h->ws.k1_status = (unsigned long long*)(b + o_k1s);
  h->ws.bfill = (int32_t*)(b + o_bf);
  h->ws.k3_status = (unsigned long long*)(b + o_k3s);
  h->ws.rbase = (int32_t*)(b + o_rb);
  h->ws.brow = (uint16_t*)(b + o_br);
  h->ws.bval = (uint32_t*)(b + o_bv);
  h->ws.hot_rows = (const int32_t*)(b + o_hr);
  h->ws.rowidx_k2 = nullptr;
  h->ws.hot_start = (const int32_t*)(b + o_hs);
  h->ws.hot_val = (uint32_t*)(b + o_hv);
  h->ws.hot_touch = (uint32_t*)(b + o_ht);
  h->ws.nhot = 0;

  int rc = SPMSPV_OK;
  do {
    if ((e = cudaMemset(h->ws_base, 0, zero_bytes)) != cudaSuccess) { rc = cuda_fail(e, "memset"); break; }
    // bucket regions: the nonzeros of A in each fine row range, prefix-summed
    int32_t* d_counts = nullptr;
    unsigned int* d_bad = nullptr;
    if ((e = cudaMalloc(&d_counts, sizeof(int32_t) * (size_t)h->nb_fine + 16)) != cudaSuccess) {
      rc = fail(SPMSPV_ERR_OOM, "bucket count scratch: %s", cudaGetErrorString(e));
      break;
    }
    d_bad = (unsigned int*)(d_counts + h->nb_fine);
    cudaMemset(d_counts, 0, sizeof(int32_t) * (size_t)h->nb_fine + 16);
    if (nnz > 0 && (e = launch_bucket_sizes(h->A, h->lwb_lo, h->nb_fine, d_counts, d_bad, 0)) != cudaSuccess) {
      cudaFree(d_counts);
      rc = cuda_fail(e, "bucket size launch");
      break;
    }
    std::vector<int32_t> counts((size_t)h->nb_fine + 4, 0);
    e = cudaMemcpy(counts.data(), d_counts, sizeof(int32_t) * (size_t)h->nb_fine + 16,
                   cudaMemcpyDeviceToHost);
    cudaFree(d_counts);
    if (e != cudaSuccess) { rc = cuda_fail(e, "bucket size copy"); break; }
    unsigned int bad = 0;
    memcpy(&bad, counts.data() + h->nb_fine, sizeof(bad));
    if (bad) { rc = fail(SPMSPV_ERR_INDEX, "%u row ids outside [0, m)", bad); break; }
    std::vector<int32_t> rbase((size_t)h->nb_fine + 1, 0);
    int64_t acc = 0;
    for (int i = 0; i < h->nb_fine; ++i) {
      rbase[i] = (int32_t)acc;
      acc += counts[i];
    }
    rbase[h->nb_fine] = (int32_t)acc;
    if (acc != nnz) { rc = fail(SPMSPV_ERR_ARG, "row histogram %lld != nnz %lld", (long long)acc, (long long)nnz); break; }
    if ((e = cudaMemcpy(h->ws.rbase, rbase.data(), sizeof(int32_t) * rbase.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess) { rc = cuda_fail(e, "rbase copy"); break; }
    // hub rows: the (at most HOT_MAX) rows of largest degree with at least
    // HOT_MIN_DEG nonzeros; their products are combined per K2 tile
    if ((rc = select_hot_rows(h)) != SPMSPV_OK) break;
    // row ids ascending in every column? (lets the pull BFS stop at the first hit)
    {
      int32_t* d_u = nullptr;
      if ((e = cudaMalloc(&d_u, sizeof(int32_t))) != cudaSuccess) {
        rc = fail(SPMSPV_ERR_OOM, "scratch: %s", cudaGetErrorString(e));
        break;
      }
      cudaMemset(d_u, 0, sizeof(int32_t));
      int32_t u = 1;
      e = launch_rows_unsorted(h->A, d_u, 0);
      if (e == cudaSuccess) e = cudaMemcpy(&u, d_u, sizeof(int32_t), cudaMemcpyDeviceToHost);
      cudaFree(d_u);
      if (e != cudaSuccess) { rc = cuda_fail(e, "row order check"); break; }
      h->rows_sorted = u == 0;
    }
    // pull direction buffers (the CSC doubles as CSR only for a symmetric pattern)
    if ((flags & SPMSPV_CSC_PATTERN_SYMMETRIC) && m == n && !jc) {
      if ((e = alloc_pull_buffers(h)) != cudaSuccess) {
        rc = fail(SPMSPV_ERR_OOM, "pull buffers: %s", cudaGetErrorString(e));
        break;
      }
    }
    // default schedule state
    DevState st0;
    memset(&st0, 0, sizeof(st0));
    st0.q = 2 * QF;  // schedule 5 (the default)
    st0.lwb = h->lwb_lo + 2;
    if ((e = cudaMemcpy(h->ws.st, &st0, sizeof(st0), cudaMemcpyHostToDevice)) != cudaSuccess) {
      rc = cuda_fail(e, "state init");
      break;
    }
    // dense accumulator of the direct (+,*) form, every row -0.0
    if (m <= DIRECT_M_MAX) {
      if ((e = cudaMalloc(&h->ws.ydense, sizeof(float) * (size_t)m)) != cudaSuccess) {
        rc = fail(SPMSPV_ERR_OOM, "dense accumulator: %s", cudaGetErrorString(e));
        break;
      }
      if ((e = launch_fill_u32(reinterpret_cast<uint32_t*>(h->ws.ydense), m, 0x80000000u, 0)) != cudaSuccess ||
          (e = cudaDeviceSynchronize()) != cudaSuccess) {
        rc = cuda_fail(e, "dense accumulator fill");
        break;
      }
    }
    h->k2_smem = k2_smem_bytes(h->nb_fine, h->ws.nhot > 0);
    h->k3_smem_max = k3_smem_bytes(lwb_hi);
    // the attribute is per kernel, not per handle: always allow the largest
    // layout any handle can need, so that a later handle never lowers it
    if ((e = set_kernel_attributes(k2_smem_bytes(NB_K2_MAX, true), k3_smem_bytes(LWB_MAX))) !=
        cudaSuccess) {
      rc = cuda_fail(e, "kernel attributes");
      break;
    }
    const int k2_bps = k2_blocks_per_sm(kPlusTimes, h->k2_smem);
    h->k2_grid = h->sm_count * k2_bps;
    for (int i = 0; i < 3; ++i) h->k3_bps[i] = k3_blocks_per_sm(kPlusTimes, k3_smem_bytes(h->lwb_lo + i));
    h->k1_grid_max = h->sm_count * 4;
    h->k1_grid_dev = h->sm_count * 2;
    h->default_sched = 5;  // push, 4096-product tiles, widest buckets: the fastest
                           // single schedule at R-MAT s22 with nnz(x) = 10^6
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) { rc = cuda_fail(e, "create"); break; }
  } while (0);
  if (rc != SPMSPV_OK) {
    release_extras(h);
    cudaFree(h->rowidx_k2);
    cudaFree(h->ws.ydense);
    cudaFree(h->ws_base);
    cudaFree(h->dcsc_aux);
    h->magic = 0;
    delete h;
    return rc;
  }
  *out = h;
  return SPMSPV_OK;
}

}  // namespace spmspv

extern "C" {

int spmspv_create_csc(spmspv_handle** out, int32_t m, int32_t n, int64_t nnz, const int32_t* colptr,
                      const int32_t* rowidx, const void* val, int val_type, uint32_t flags) {
  return create_impl(out, m, n, nnz, colptr, rowidx, val, val_type, flags, nullptr, 0);
}

int spmspv_dcsc_index(int32_t n, int32_t nzc, const int32_t* jc, int32_t* aux, int64_t aux_capacity,
                      int64_t* aux_len, int32_t* shift) {
  if (n < 1 || nzc < 0 || nzc > n) return fail(SPMSPV_ERR_ARG, "need n >= 1 and 0 <= nzc <= n");
  if (nzc > 0 && !jc) return fail(SPMSPV_ERR_ARG, "jc is NULL");
  std::vector<int32_t> a;
  int s = 0;
  int rc = dcsc_index_host(n, 0, nzc, jc, nullptr, a, s);
  if (rc != SPMSPV_OK) return rc;
  if (aux_len) *aux_len = (int64_t)a.size();
  if (shift) *shift = s;
  if (aux && aux_capacity > 0)
    memcpy(aux, a.data(), sizeof(int32_t) * (size_t)std::min<int64_t>(aux_capacity, (int64_t)a.size()));
  return SPMSPV_OK;
}

int spmspv_create_dcsc(spmspv_handle** out, int32_t m, int32_t n, int64_t nnz, int32_t nzc,
                       const int32_t* jc, const int32_t* cp, const int32_t* rowidx, const void* val,
                       int val_type, uint32_t flags) {
  if (nzc < 0 || nzc > n) return fail(SPMSPV_ERR_ARG, "nzc = %d outside [0, n]", nzc);
  if (nzc > 0 && !jc) return fail(SPMSPV_ERR_ARG, "jc is NULL");
  if (!cp) return fail(SPMSPV_ERR_ARG, "cp is NULL");
  // with nzc = 0 the (never read) jc stays non-NULL so that the handle is a DCSC one
  return create_impl(out, m, n, nnz, cp, rowidx, val, val_type, flags, jc ? jc : cp, nzc);
}

int spmspv_destroy(spmspv_handle* h) {
  if (!h || h->magic != kHandleMagic) return fail(SPMSPV_ERR_STATE, "invalid or destroyed handle");
  cudaDeviceSynchronize();
  if (h->prof) {
    double tmp[SPMSPV_NUM_STAGES];
    spmspv_profile_end(h, tmp, SPMSPV_NUM_STAGES, nullptr);
  }
  release_bfs_graphs(h);
  release_batch(h);
  release_k6(h);
  release_cc(h);
  release_mis(h);
  release_mcm(h);
  release_sortx(h);
  release_tune(h);
  release_hostio(h);
  release_extras(h);
  cudaFree(h->rowidx_k2);
  cudaFree(h->sel_w);
  cudaFree(h->ws.ydense);
  cudaFree(h->ws_base);
  cudaFree(h->dcsc_aux);
  h->magic = 0;
  delete h;
  return SPMSPV_OK;
}

int spmspv_run(spmspv_handle* h, int semiring, const int32_t* x_idx, const void* x_val,
               int32_t nnz_x, const uint32_t* mask, uint32_t opts, int32_t* y_idx, void* y_val,
               int32_t y_capacity, int32_t* d_nnz_y, spmspv_stream_t stream) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (semiring < 0 || semiring > 2) return fail(SPMSPV_ERR_ARG, "unknown semiring %d", semiring);
  if (nnz_x < 0 || nnz_x > h->A.n) return fail(SPMSPV_ERR_ARG, "nnz_x = %d outside [0, n]", nnz_x);
  if (nnz_x > 0 && !x_idx) return fail(SPMSPV_ERR_ARG, "x_idx is NULL");
  if (nnz_x > 0 && semiring != SPMSPV_OR_AND_BOOL && !x_val)
    return fail(SPMSPV_ERR_ARG, "x_val is NULL");
  if (y_capacity < 0) return fail(SPMSPV_ERR_ARG, "y_capacity < 0");
  if (y_capacity > 0 && !y_idx) return fail(SPMSPV_ERR_ARG, "y_idx is NULL");
  if (y_capacity > 0 && semiring != SPMSPV_OR_AND_BOOL && !y_val)
    return fail(SPMSPV_ERR_ARG, "y_val is NULL");
  if (!d_nnz_y) return fail(SPMSPV_ERR_ARG, "d_nnz_y is NULL");
  if ((opts & SPMSPV_SCHED_FORCE) && SPMSPV_SCHED_ID(opts) >= SPMSPV_NUM_SCHEDULES)
    return fail(SPMSPV_ERR_ARG, "schedule id %u out of range", SPMSPV_SCHED_ID(opts));
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  if (nnz_x == 0) {
    cudaError_t e = cudaMemsetAsync(d_nnz_y, 0, sizeof(int32_t), s);
    h->last_empty = 1;
    return e == cudaSuccess ? SPMSPV_OK : cuda_fail(e, "memset nnz_y");
  }
  h->last_empty = 0;
  if ((opts & SPMSPV_SORT_X) && nnz_x > 1) {
    if ((rc = sort_x(h, x_idx, (const uint32_t*)x_val, nnz_x, s)) != SPMSPV_OK) return rc;
    x_idx = h->sx_idx;
    x_val = x_val ? (const void*)h->sx_val : nullptr;
  }
  const int mask_comp = (opts & SPMSPV_MASK_COMPLEMENT) ? 1 : 0;
  h->plus_direct = (opts & SPMSPV_BUCKETS_ONLY) ? 0 : 1;
  // x(j) = j (a BFS frontier) and ascending row ids: a pull row may stop at
  // its first frontier neighbour, the smallest
  const int early_exit = (opts & SPMSPV_X_IDS) && semiring == SPMSPV_MIN_SELECT2ND_I32 && h->rows_sorted ? 1 : 0;
  if (opts & SPMSPV_SCHED_AUTO) {
    if (!h->sel_ready) return fail(SPMSPV_ERR_STATE, "no selector weights loaded or trained");
    return run_auto(h, semiring, x_idx, (const uint32_t*)x_val, nnz_x, mask, mask_comp, y_idx,
                    (uint32_t*)y_val, y_capacity, d_nnz_y, s, early_exit);
  }
  int sid = h->default_sched;
  if (opts & SPMSPV_SCHED_FORCE) sid = (int)SPMSPV_SCHED_ID(opts);
  Sched sc = decode_schedule(h, sid);
  if (sc.dir == 1) {
    rc = run_pull_if_available(h, semiring, x_idx, (const uint32_t*)x_val, nnz_x, mask, mask_comp,
                               sc, y_idx, (uint32_t*)y_val, y_capacity, d_nnz_y, s, early_exit);
    if (rc != -1) return rc;
    sc.dir = 0;  // no row access to A: the push form of the same schedule
    sc.id = sc.id % 6;
  }
  h->k1_mask = (opts & SPMSPV_WITH_FEATURES) ? mask : nullptr;
  rc = run_push(h, semiring, x_idx, (const uint32_t*)x_val, nnz_x, nullptr, mask, mask_comp, sc,
                y_idx, (uint32_t*)y_val, y_capacity, d_nnz_y, false, nullptr, s);
  h->k1_mask = nullptr;
  return rc;
}

int spmspv_device_status(spmspv_handle* h, uint32_t* flags) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!flags) return fail(SPMSPV_ERR_ARG, "flags is NULL");
  cudaError_t e = cudaStreamSynchronize(h->last_stream);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  uint32_t v = 0;
  e = cudaMemcpy(&v, &h->ws.st->status, sizeof(v), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "status copy");
  uint32_t z = 0;
  e = cudaMemcpy(&h->ws.st->status, &z, sizeof(z), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "status clear");
  v |= batch_collect_status(h, &e);  // the batched lanes' own workspaces
  if (e != cudaSuccess) return cuda_fail(e, "lane status");
  *flags = v & (SPMSPV_DEV_CAPACITY | SPMSPV_DEV_TIMEOUT | ST_INDEX | ST_BOUND);
  return SPMSPV_OK;
}

int spmspv_last_work(spmspv_handle* h, int64_t* work) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!work) return fail(SPMSPV_ERR_ARG, "work is NULL");
  cudaError_t e = cudaStreamSynchronize(h->last_stream);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  if (h->last_empty) {
    *work = 0;
    return SPMSPV_OK;
  }
  int32_t W = 0;
  e = cudaMemcpy(&W, &h->ws.st->W, sizeof(W), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "work copy");
  *work = W;
  return SPMSPV_OK;
}

int spmspv_profile_begin(spmspv_handle* h) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!h->prof) h->prof = new ProfileLog();
  return SPMSPV_OK;
}

int spmspv_profile_end(spmspv_handle* h, double* stage_ms, int32_t n_stages, int32_t* n_calls) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!stage_ms || n_stages < 0) return fail(SPMSPV_ERR_ARG, "stage_ms is NULL");
  for (int i = 0; i < n_stages; ++i) stage_ms[i] = 0.0;
  ProfileLog* log = (ProfileLog*)h->prof;
  if (n_calls) *n_calls = log ? (int32_t)log->size() : 0;
  if (!log) return SPMSPV_OK;
  h->prof = nullptr;
  cudaError_t err = cudaSuccess;
  for (ProfileCall& c : *log) {
    for (size_t i = 0; i + 1 < c.events.size(); ++i) {
      cudaError_t e = cudaEventSynchronize(c.events[i + 1]);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, c.events[i], c.events[i + 1]);
      if (e != cudaSuccess) err = e;
      const int st = c.stages[i];
      if (st >= 0 && st < n_stages) stage_ms[st] += ms;
    }
    for (cudaEvent_t e : c.events) cudaEventDestroy(e);
  }
  delete log;
  return err == cudaSuccess ? SPMSPV_OK : cuda_fail(err, "profile events");
}

}  // extern "C"
