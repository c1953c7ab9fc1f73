// Device side of the learned schedule selector, shared by the work scan
// (which runs the choice in its last CTA) and the selector's own kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "spmspv_internal.cuh"

namespace spmspv {

constexpr int SEL_IN = 6, SEL_H = 32, SEL_OUT = 12;
constexpr int SEL_OW1 = 0, SEL_OB1 = SEL_OW1 + SEL_H * SEL_IN, SEL_OW2 = SEL_OB1 + SEL_H,
              SEL_OB2 = SEL_OW2 + SEL_H * SEL_H, SEL_OW3 = SEL_OB2 + SEL_H,
              SEL_OB3 = SEL_OW3 + SEL_OUT * SEL_H, SEL_NWEIGHT = SEL_OB3 + SEL_OUT;  // 1676
constexpr int SEL_OMEAN = SEL_NWEIGHT, SEL_OSCALE = SEL_OMEAN + SEL_IN, SEL_NPARAM = SEL_OSCALE + SEL_IN;
static_assert(SEL_NWEIGHT == 1676, "MLP size");

// One warp evaluates the network for one normalised input; lane j holds
// hidden unit j.  Returns the prediction of output `lane` (lanes < 12).
__device__ __forceinline__ float sel_forward_warp(const float* __restrict__ w, const float* xin,
                                                  float* h1o, float* h2o) {
  const int lane = threadIdx.x & 31;
  float a1 = w[SEL_OB1 + lane];
#pragma unroll
  for (int k = 0; k < SEL_IN; ++k) a1 += w[SEL_OW1 + lane * SEL_IN + k] * xin[k];
  const float h1 = fmaxf(a1, 0.f);
  float a2 = w[SEL_OB2 + lane];
#pragma unroll
  for (int k = 0; k < SEL_H; ++k) a2 += w[SEL_OW2 + lane * SEL_H + k] * __shfl_sync(0xffffffffu, h1, k);
  const float h2 = fmaxf(a2, 0.f);
  float o = 0.f;
  const int r = lane < SEL_OUT ? lane : 0;
  o = w[SEL_OB3 + r];
#pragma unroll
  for (int k = 0; k < SEL_H; ++k) o += w[SEL_OW3 + r * SEL_H + k] * __shfl_sync(0xffffffffu, h2, k);
  if (h1o) *h1o = h1;
  if (h2o) *h2o = h2;
  return o;
}

// bfs: the mask is the BFS visited set, whose population is the count of
// vertices reached so far (no pass over the bitmap needed).
// The six features from the call's counts: f = nnz(x), W = products, fc =
// x entries with a non-empty column, the largest selected column, and the
// number of rows set in the mask (in BFS, the vertices reached so far).
__device__ __forceinline__ void sel_features_of(int32_t f_i, int32_t W_i, int32_t fc_i, int32_t maxdeg,
                                                int32_t maskcnt, int32_t m, int32_t n, int64_t nnz,
                                                float* x) {
  const float f = (float)f_i, W = (float)W_i;
  const float fc = (float)max(fc_i, 1);
  x[0] = log2f(1.f + f);
  x[1] = log2f(1.f + W);
  x[2] = W > 0.f ? (float)maxdeg * fc / W : 0.f;
  x[3] = (float)maskcnt / (float)m;
  x[4] = log2f((float)m);
  x[5] = (float)((double)nnz / (double)n);
}

__device__ __forceinline__ void sel_features(const DevState* st, int32_t m, int32_t n, int64_t nnz,
                                             int bfs, float* x) {
  // L2 reads: other CTAs of the same launch may have written these
  sel_features_of(__ldcg(&st->f), __ldcg(&st->W), __ldcg(&st->fc), __ldcg(&st->maxdeg),
                  bfs ? __ldcg(&st->nvisited) : __ldcg(&st->maskcnt), m, n, nnz, x);
}

// The schedule the network picks for raw features x (one full warp; every
// lane gets the id): normalise, evaluate, argmin over the allowed outputs
// (ties to the smaller id).
__device__ __forceinline__ int sel_pick_warp(const float* __restrict__ w, const float* xraw, int allow_pull) {
  float x[SEL_IN];
#pragma unroll
  for (int k = 0; k < SEL_IN; ++k) x[k] = (xraw[k] - w[SEL_OMEAN + k]) * w[SEL_OSCALE + k];
  const float o = sel_forward_warp(w, x, nullptr, nullptr);
  const int lane = threadIdx.x & 31;
  const bool ok = lane < SEL_OUT && (allow_pull || lane < 6);
  float best = ok ? o : INFINITY;
  int bi = ok ? lane : 64;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, off);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
    if (ob < best || (ob == best && oi < bi)) {
      best = ob;
      bi = oi;
    }
  }
  return bi < SEL_OUT ? bi : 4;
}

// The direction-optimizing rule with two fixed thresholds (Beamer, Asanovic
// and Patterson, "Direction-Optimizing Breadth-First Search", SC 2012, with
// their alpha = 14 and beta = 24), the baseline the learned selector is
// measured against: from push to pull once the frontier's edges exceed the
// unvisited vertices' edges / alpha, back to push once the frontier holds
// fewer than n / beta vertices.  Returns 1 for pull.
constexpr int RULE_ALPHA = 14, RULE_BETA = 24;
__device__ __forceinline__ int rule_direction(int prev_dir, int32_t f, long long W, long long edges_unvisited,
                                              int32_t n, int allow_pull) {
  if (!allow_pull) return 0;
  if (prev_dir == 0) return W * RULE_ALPHA > edges_unvisited ? 1 : 0;
  return (long long)f * RULE_BETA < (long long)n ? 0 : 1;
}

// Device-side choice for this call, run by one full warp: features -> MLP ->
// argmin over the allowed schedules -> state (direction, quantum, bucket
// width).  Inside a graph, the two conditional handles (when given) select
// the push or the pull branch of the level.
__device__ __forceinline__ void sel_choose_warp(const float* __restrict__ w, DevState* st, int32_t m,
                                                int32_t n, int64_t nnz, const SelArgs& a) {
  const int lwb_lo = a.lwb_lo;
  // a BFS level small enough for the direct form stays push: there it costs
  // a few microseconds, less than any pull, whatever decides the others
  const bool small_bfs = a.bfs && a.direct_max > 0 && __ldcg(&st->W) <= a.direct_max;
  if (a.rule) {  // the baseline rule: the default push schedule, or pull
    const long long W = __ldcg(&st->W);
    const long long seen = __ldcg(&st->edges_seen) + W;
    const int dir = small_bfs ? 0 : rule_direction(__ldcg(&st->dir), __ldcg(&st->f), W, nnz - seen, n, a.allow_pull);
    if ((threadIdx.x & 31) == 0) {
      st->edges_seen = seen;
      const int id = dir ? 11 : 5;
      st->sched = id;
      st->dir = dir;
      st->q = 2 * QF;
      st->lwb = lwb_lo + 2;
    }
    return;
  }
  float x[SEL_IN];
  sel_features(st, m, n, nnz, a.bfs, x);
  if ((threadIdx.x & 31) == 0) {  // kept for spmspv_last_features
#pragma unroll
    for (int k = 0; k < SEL_IN; ++k) st->feat[k] = x[k];
    st->feat_dev = 1;
  }
#pragma unroll
  for (int k = 0; k < SEL_IN; ++k) x[k] = (x[k] - w[SEL_OMEAN + k]) * w[SEL_OSCALE + k];
  const float o = sel_forward_warp(w, x, nullptr, nullptr);
  const int lane = threadIdx.x & 31;
  const bool ok = lane < SEL_OUT && (a.allow_pull || lane < 6);
  float best = ok ? o : INFINITY;
  int bi = ok ? lane : 64;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, off);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
    if (ob < best || (ob == best && oi < bi)) {
      best = ob;
      bi = oi;
    }
  }
  if (lane == 0) {
    int id = bi < SEL_OUT ? bi : 4;
    if (small_bfs && id >= 6) id -= 6;  // the push schedule of the same quantum and width
    st->sched = id;
    st->dir = id / 6;
    st->q = ((id / 3) % 2) ? 2 * QF : QF;
    st->lwb = lwb_lo + id % 3;
    if (a.use_cond) {
      cudaGraphSetConditional(a.c_push, id / 6 == 0 ? 1u : 0u);
      cudaGraphSetConditional(a.c_pull, id / 6 == 1 ? 1u : 0u);
    }
  }
}

}  // namespace spmspv
