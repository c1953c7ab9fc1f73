// Learned schedule selector: a 6 -> 32 -> 32 -> 12 FP32 MLP (ReLU) that
// predicts the log run time of each of the 12 schedules (3 bucket widths x
// 2 work quanta x {push, pull}) from features of the call, and picks the
// schedule with the smallest prediction.  It never changes results, only
// which kernels and tile/bucket sizes compute them.  The paper has no such
// component; it answers the paper's open question of when to switch to a
// matrix-driven algorithm (Sec. V).
//
// Features (computed on the device from the work scan's outputs):
//   0 log2(1 + nnz(x))        1 log2(1 + W)       2 max column length / mean
//   3 masked-row fraction     4 log2(m)           5 nnz(A) / n
//
// Weight layout (float, SEL_NPARAM): W1[32][6] b1[32] W2[32][32] b2[32]
// W3[12][32] b3[12], then the feature normalisation mean[6] and scale[6].
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "handle.cuh"
#include "selector_dev.cuh"
#include "spmspv_internal.cuh"

namespace spmspv {


// Training: mean squared error over the valid (sample, schedule) targets.
// One warp per sample; each lane accumulates the gradient of the weights it
// owns (column `lane` of W2 and W3, row `lane` of W1, its biases) in registers
// over the warp's samples, then adds it to the global gradient once.
__global__ void k_sel_grad(const float* __restrict__ w, const float* __restrict__ feats,
                           const float* __restrict__ target, const uint8_t* __restrict__ valid,
                           const int32_t* __restrict__ order, int32_t n0, int32_t nb,
                           float* __restrict__ grad, float* __restrict__ loss) {
  const int lane = threadIdx.x & 31;
  const int warps = blockDim.x / 32;
  float gW3[SEL_OUT], gW2[SEL_H], gW1[SEL_IN], gb1 = 0.f, gb2 = 0.f, gb3 = 0.f, lsum = 0.f;
#pragma unroll
  for (int i = 0; i < SEL_OUT; ++i) gW3[i] = 0.f;
#pragma unroll
  for (int i = 0; i < SEL_H; ++i) gW2[i] = 0.f;
#pragma unroll
  for (int i = 0; i < SEL_IN; ++i) gW1[i] = 0.f;
  for (int sidx = blockIdx.x * warps + (threadIdx.x >> 5); sidx < nb; sidx += gridDim.x * warps) {
    const int sm = order ? order[n0 + sidx] : n0 + sidx;
    float x[SEL_IN];
#pragma unroll
    for (int k = 0; k < SEL_IN; ++k)
      x[k] = (feats[(size_t)sm * SEL_IN + k] - w[SEL_OMEAN + k]) * w[SEL_OSCALE + k];
    float h1, h2;
    const float o = sel_forward_warp(w, x, &h1, &h2);
    float d_o = 0.f;
    if (lane < SEL_OUT) {
      const bool v = valid ? valid[(size_t)sm * SEL_OUT + lane] != 0 : true;
      if (v) {
        const float diff = o - target[(size_t)sm * SEL_OUT + lane];
        d_o = 2.f * diff;
        lsum += diff * diff;
      }
    }
    gb3 += d_o;
    // layer 3: dW3[o][lane] = d_o[o] * h2[lane]; d_h2[lane] = sum_o W3[o][lane] d_o[o]
    float dh2 = 0.f;
#pragma unroll
    for (int oo = 0; oo < SEL_OUT; ++oo) {
      const float dor = __shfl_sync(0xffffffffu, d_o, oo);
      gW3[oo] += dor * h2;
      dh2 += w[SEL_OW3 + oo * SEL_H + lane] * dor;
    }
    if (h2 <= 0.f) dh2 = 0.f;
    gb2 += dh2;
    // layer 2: dW2[j][lane] = d_h2[j] * h1[lane]; d_h1[lane] = sum_j W2[j][lane] d_h2[j]
    float dh1 = 0.f;
#pragma unroll
    for (int j = 0; j < SEL_H; ++j) {
      const float dj = __shfl_sync(0xffffffffu, dh2, j);
      gW2[j] += dj * h1;
      dh1 += w[SEL_OW2 + j * SEL_H + lane] * dj;
    }
    if (h1 <= 0.f) dh1 = 0.f;
    gb1 += dh1;
    // layer 1: dW1[lane][k] = d_h1[lane] * x[k]
#pragma unroll
    for (int k = 0; k < SEL_IN; ++k) gW1[k] += dh1 * x[k];
  }
#pragma unroll
  for (int oo = 0; oo < SEL_OUT; ++oo)
    if (gW3[oo] != 0.f) atomicAdd(&grad[SEL_OW3 + oo * SEL_H + lane], gW3[oo]);
#pragma unroll
  for (int j = 0; j < SEL_H; ++j)
    if (gW2[j] != 0.f) atomicAdd(&grad[SEL_OW2 + j * SEL_H + lane], gW2[j]);
#pragma unroll
  for (int k = 0; k < SEL_IN; ++k)
    if (gW1[k] != 0.f) atomicAdd(&grad[SEL_OW1 + lane * SEL_IN + k], gW1[k]);
  if (gb1 != 0.f) atomicAdd(&grad[SEL_OB1 + lane], gb1);
  if (gb2 != 0.f) atomicAdd(&grad[SEL_OB2 + lane], gb2);
  if (lane < SEL_OUT && gb3 != 0.f) atomicAdd(&grad[SEL_OB3 + lane], gb3);
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0 && loss && lsum != 0.f) atomicAdd(loss, lsum);
}

// Adam step on the 1676 weights (the normalisation is not trained).
__global__ void k_sel_adam(float* __restrict__ w, const float* __restrict__ grad, float* __restrict__ mom,
                           float* __restrict__ vel, float scale, float lr, float b1, float b2,
                           float b1t, float b2t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= SEL_NWEIGHT) return;
  const float g = grad[i] * scale;
  const float m1 = b1 * mom[i] + (1.f - b1) * g;
  const float v1 = b2 * vel[i] + (1.f - b2) * g * g;
  mom[i] = m1;
  vel[i] = v1;
  w[i] -= lr * (m1 / (1.f - b1t)) / (sqrtf(v1 / (1.f - b2t)) + 1e-8f);
}

static int ensure_sel_buffer(spmspv_handle* h) {
  if (h->sel_w) return SPMSPV_OK;
  cudaError_t e = cudaMalloc(&h->sel_w, sizeof(float) * SEL_NPARAM);
  if (e != cudaSuccess) {
    h->sel_w = nullptr;
    return fail(SPMSPV_ERR_OOM, "selector weights: %s", cudaGetErrorString(e));
  }
  return SPMSPV_OK;
}

}  // namespace spmspv

using namespace spmspv;

extern "C" int spmspv_selector_set(spmspv_handle* h, const float* params, int32_t n) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!params || n != SEL_NPARAM) return fail(SPMSPV_ERR_ARG, "expected %d selector parameters", SEL_NPARAM);
  if ((rc = ensure_sel_buffer(h)) != SPMSPV_OK) return rc;
  cudaError_t e = cudaMemcpy(h->sel_w, params, sizeof(float) * SEL_NPARAM, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "selector weights copy");
  h->sel_ready = 1;
  return SPMSPV_OK;
}

// Parameters from a weights file: a JSON object whose "params" member is an
// array of SPMSPV_SELECTOR_NPARAM numbers (the file selector.py writes; any
// other members, such as "nparam" and "meta", are ignored here).  The parse
// is a plain scan: find the "params" key, then read numbers between '[' and
// ']' with strtod.
static int read_selector_file(const char* path, std::vector<float>& out) {
  FILE* fp = fopen(path, "rb");
  if (!fp) return fail(SPMSPV_ERR_ARG, "cannot open selector weights file %s", path);
  std::string text;
  char buf[65536];
  size_t got;
  while ((got = fread(buf, 1, sizeof(buf), fp)) > 0) text.append(buf, got);
  fclose(fp);
  const size_t key = text.find("\"params\"");
  if (key == std::string::npos) return fail(SPMSPV_ERR_ARG, "%s has no \"params\" member", path);
  size_t i = text.find('[', key);
  if (i == std::string::npos) return fail(SPMSPV_ERR_ARG, "%s: \"params\" is not an array", path);
  ++i;
  out.clear();
  for (;;) {
    while (i < text.size() && (text[i] == ' ' || text[i] == '\n' || text[i] == '\r' || text[i] == '\t' ||
                               text[i] == ','))
      ++i;
    if (i >= text.size()) return fail(SPMSPV_ERR_ARG, "%s: unterminated \"params\" array", path);
    if (text[i] == ']') break;
    char* end = nullptr;
    const double v = strtod(text.c_str() + i, &end);
    if (end == text.c_str() + i) return fail(SPMSPV_ERR_ARG, "%s: not a number at byte %zu", path, i);
    out.push_back((float)v);
    i = (size_t)(end - text.c_str());
  }
  if ((int)out.size() != SEL_NPARAM)
    return fail(SPMSPV_ERR_ARG, "%s holds %zu selector parameters, expected %d", path, out.size(), SEL_NPARAM);
  return SPMSPV_OK;
}

extern "C" int spmspv_selector_load(spmspv_handle* h, const char* path) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!path) return fail(SPMSPV_ERR_ARG, "path is NULL");
  std::vector<float> p;
  if ((rc = read_selector_file(path, p)) != SPMSPV_OK) return rc;
  return spmspv_selector_set(h, p.data(), (int32_t)p.size());
}

extern "C" int spmspv_selector_get(spmspv_handle* h, float* params, int32_t n) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!params || n != SEL_NPARAM) return fail(SPMSPV_ERR_ARG, "expected %d selector parameters", SEL_NPARAM);
  if (!h->sel_ready) return fail(SPMSPV_ERR_STATE, "no selector weights");
  cudaError_t e = cudaMemcpy(params, h->sel_w, sizeof(float) * SEL_NPARAM, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? SPMSPV_OK : cuda_fail(e, "selector weights copy");
}

extern "C" int spmspv_last_features(spmspv_handle* h, float* feats) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!feats) return fail(SPMSPV_ERR_ARG, "feats is NULL");
  cudaError_t e = cudaStreamSynchronize(h->last_stream);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  DevState st;
  if ((e = cudaMemcpy(&st, h->ws.st, sizeof(st), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "state copy");
  if (st.feat_dev) {  // the features the selector itself evaluated in this call
    for (int k = 0; k < 6; ++k) feats[k] = st.feat[k];
    return SPMSPV_OK;
  }
  const double f = st.f, W = st.W, fc = st.fc > 0 ? st.fc : 1;
  feats[0] = (float)std::log2(1.0 + f);
  feats[1] = (float)std::log2(1.0 + W);
  feats[2] = W > 0 ? (float)(st.last_maxdeg * fc / W) : 0.f;
  feats[3] = (float)st.last_maskcnt / (float)h->A.m;
  feats[4] = (float)std::log2((double)h->A.m);
  feats[5] = (float)((double)h->A.nnz / (double)h->A.n);
  return SPMSPV_OK;
}

extern "C" int spmspv_last_schedule(spmspv_handle* h, int32_t* sched) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!sched) return fail(SPMSPV_ERR_ARG, "sched is NULL");
  cudaError_t e = cudaStreamSynchronize(h->last_stream);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  DevState st;
  if ((e = cudaMemcpy(&st, h->ws.st, sizeof(st), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "state copy");
  *sched = st.sched;
  return SPMSPV_OK;
}

/*
 * Gradient of the mean squared error over the valid targets at the current
 * weights (for checking the kernels against a CPU reference).
 */
extern "C" int spmspv_selector_grad(spmspv_handle* h, const float* feats, const float* target,
                                    const uint8_t* valid, int32_t n, float* grad_host,
                                    float* loss_host) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!h->sel_ready) return fail(SPMSPV_ERR_STATE, "no selector weights");
  if (!feats || !target || n < 1 || !grad_host) return fail(SPMSPV_ERR_ARG, "bad arguments");
  float* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(float) * (SEL_NWEIGHT + 1));
  if (e != cudaSuccess) return fail(SPMSPV_ERR_OOM, "gradient buffer");
  cudaMemset(d, 0, sizeof(float) * (SEL_NWEIGHT + 1));
  const int grid = std::min(h->sm_count, (n + 7) / 8);
  k_sel_grad<<<grid, 256>>>(h->sel_w, feats, target, valid, nullptr, 0, n, d, d + SEL_NWEIGHT);
  e = cudaGetLastError();
  std::vector<float> tmp(SEL_NWEIGHT + 1);
  if (e == cudaSuccess) e = cudaMemcpy(tmp.data(), d, sizeof(float) * (SEL_NWEIGHT + 1), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "selector gradient");
  memcpy(grad_host, tmp.data(), sizeof(float) * SEL_NWEIGHT);
  if (loss_host) *loss_host = tmp[SEL_NWEIGHT];
  return SPMSPV_OK;
}

/*
 * Mini-batch Adam training of the selector on the device.  feats [n][6] raw
 * features, target [n][12] log run times, valid [n][12] (NULL: all valid);
 * device pointers.  The normalisation (mean/scale) is taken from the data;
 * the weights start from the handle's current ones when present, else from a
 * seeded He initialisation.  loss_host (may be NULL) receives the mean loss of
 * each epoch.
 */
extern "C" int spmspv_selector_train(spmspv_handle* h, const float* feats, const float* target,
                                     const uint8_t* valid, int32_t n, int32_t epochs, int32_t batch,
                                     float lr, uint64_t seed, float* loss_host) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!feats || !target || n < 1 || epochs < 0 || batch < 1 || !(lr > 0.f))
    return fail(SPMSPV_ERR_ARG, "bad training arguments");
  if ((rc = ensure_sel_buffer(h)) != SPMSPV_OK) return rc;
  std::vector<float> hf((size_t)n * SEL_IN);
  cudaError_t e = cudaMemcpy(hf.data(), feats, sizeof(float) * hf.size(), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "feature copy");
  std::vector<float> p(SEL_NPARAM, 0.f);
  if (h->sel_ready) {
    e = cudaMemcpy(p.data(), h->sel_w, sizeof(float) * SEL_NPARAM, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "weights copy");
  } else {
    // He initialisation from a splitmix64 stream
    uint64_t z = seed;
    auto rnd = [&]() {
      z += 0x9E3779B97F4A7C15ULL;
      uint64_t t = z;
      t = (t ^ (t >> 30)) * 0xBF58476D1CE4E5B9ULL;
      t = (t ^ (t >> 27)) * 0x94D049BB133111EBULL;
      t ^= t >> 31;
      return ((double)(t >> 11) + 0.5) / 9007199254740992.0;
    };
    auto gauss = [&]() { return std::sqrt(-2.0 * std::log(rnd())) * std::cos(6.283185307179586 * rnd()); };
    for (int i = 0; i < SEL_H * SEL_IN; ++i) p[SEL_OW1 + i] = (float)(gauss() * std::sqrt(2.0 / SEL_IN));
    for (int i = 0; i < SEL_H * SEL_H; ++i) p[SEL_OW2 + i] = (float)(gauss() * std::sqrt(2.0 / SEL_H));
    for (int i = 0; i < SEL_OUT * SEL_H; ++i) p[SEL_OW3 + i] = (float)(gauss() * std::sqrt(1.0 / SEL_H));
  }
  // normalisation from the data
  for (int k = 0; k < SEL_IN; ++k) {
    double s = 0, s2 = 0;
    for (int32_t i = 0; i < n; ++i) {
      s += hf[(size_t)i * SEL_IN + k];
      s2 += (double)hf[(size_t)i * SEL_IN + k] * hf[(size_t)i * SEL_IN + k];
    }
    const double mean = s / n, var = s2 / n - mean * mean;
    p[SEL_OMEAN + k] = (float)mean;
    p[SEL_OSCALE + k] = (float)(var > 1e-12 ? 1.0 / std::sqrt(var) : 1.0);
  }
  e = cudaMemcpy(h->sel_w, p.data(), sizeof(float) * SEL_NPARAM, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "weights copy");
  h->sel_ready = 1;
  float* buf = nullptr;  // grad, m, v, loss
  int32_t* order = nullptr;
  if ((e = cudaMalloc(&buf, sizeof(float) * (3 * SEL_NWEIGHT + 1))) != cudaSuccess ||
      (e = cudaMalloc(&order, sizeof(int32_t) * (size_t)n)) != cudaSuccess) {
    cudaFree(buf);
    return fail(SPMSPV_ERR_OOM, "training buffers");
  }
  cudaMemset(buf, 0, sizeof(float) * (3 * SEL_NWEIGHT + 1));
  float* grad = buf;
  float* mom = buf + SEL_NWEIGHT;
  float* vel = buf + 2 * SEL_NWEIGHT;
  float* loss = buf + 3 * SEL_NWEIGHT;
  std::vector<int32_t> ord(n);
  uint64_t z = seed ^ 0xD1B54A32D192ED03ULL;
  int64_t t = 0;
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    for (int32_t i = 0; i < n; ++i) ord[i] = i;
    for (int32_t i = n - 1; i > 0; --i) {  // shuffle
      z = z * 6364136223846793005ULL + 1442695040888963407ULL;
      const int32_t j = (int32_t)((z >> 33) % (uint64_t)(i + 1));
      std::swap(ord[i], ord[j]);
    }
    cudaMemcpy(order, ord.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice);
    cudaMemset(loss, 0, sizeof(float));
    for (int32_t s0 = 0; s0 < n; s0 += batch) {
      const int32_t nb = std::min(batch, n - s0);
      cudaMemsetAsync(grad, 0, sizeof(float) * SEL_NWEIGHT);
      const int grid = std::max(1, std::min(h->sm_count, (nb + 7) / 8));
      k_sel_grad<<<grid, 256>>>(h->sel_w, feats, target, valid, order, s0, nb, grad, loss);
      ++t;
      k_sel_adam<<<(SEL_NWEIGHT + 255) / 256, 256>>>(h->sel_w, grad, mom, vel, 1.f / (float)nb, lr, 0.9f,
                                                     0.999f, (float)std::pow(0.9, (double)t),
                                                     (float)std::pow(0.999, (double)t));
    }
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if (loss_host) {
      float lv = 0.f;
      e = cudaMemcpy(&lv, loss, sizeof(float), cudaMemcpyDeviceToHost);
      loss_host[ep] = lv / (float)n;
    }
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(buf);
  cudaFree(order);
  return e == cudaSuccess ? SPMSPV_OK : cuda_fail(e, "selector training");
}

extern "C" int spmspv_default_schedule(spmspv_handle* h, int32_t* sched) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!sched) return fail(SPMSPV_ERR_ARG, "sched is NULL");
  *sched = h->default_sched;
  return SPMSPV_OK;
}
