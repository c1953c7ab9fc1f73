/*
 * Seeded synthetic sparse matrices in CSC form.
 *
 * These generators feed identical inputs to the CPU oracle and to the GPU
 * path.  They hold none of the SpMSpV arithmetic: they only draw matrices.
 * Every random number comes from a counter-based hash of (seed, stream,
 * counter), so a draw never depends on thread count or call order, and the
 * integer-only paths give the same bits on every host.
 *
 * Generators (the paper's own matrices, the University of Florida set of
 * Table IV, are not available; these stand in for its two classes):
 *  - Erdos-Renyi G(n, p) with p = d/m, the analysis model of Sec. II-A.
 *  - R-MAT (low-diameter, scale-free), symmetrised, self-loops dropped,
 *    duplicates merged, vertices relabelled by a seeded permutation.
 *  - 2D/3D grids (high-diameter), 5- or 7-point stencil without the
 *    diagonal, with a seeded fraction of undirected edges removed.
 *
 * All functions return a heap-allocated CSC through synth_csc; release it
 * with synth_free.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int64_t m, n, nnz;
  int32_t* colptr; /* n+1 */
  int32_t* rowidx; /* nnz, ascending within each column */
  float* val;      /* nnz, uniform [0,1) (NULL if not requested) */
} synth_csc;

/* splitmix64 finaliser over a combined (seed, stream, counter) key */
static inline uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ULL;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBULL;
  z ^= z >> 31;
  return z;
}

static inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t ctr) {
  uint64_t k = mix64(seed * 0x9E3779B97F4A7C15ULL + 0x632BE59BD9B4E019ULL);
  k = mix64(k ^ (stream * 0xD1B54A32D192ED03ULL + 0x8CB92BA72F3D8DD7ULL));
  return mix64(k + ctr * 0x9E3779B97F4A7C15ULL);
}

/* uniform float in [0,1) with 24 random bits */
static inline float draw_f32(uint64_t seed, uint64_t stream, uint64_t ctr) {
  return (float)(draw(seed, stream, ctr) >> 40) * (1.0f / 16777216.0f);
}

/* uniform double in (0,1] with 53 random bits */
static inline double draw_f64_open0(uint64_t seed, uint64_t stream, uint64_t ctr) {
  return ((double)(draw(seed, stream, ctr) >> 11) + 1.0) * (1.0 / 9007199254740992.0);
}

void synth_free(synth_csc* a) {
  if (!a) return;
  free(a->colptr);
  free(a->rowidx);
  free(a->val);
  a->colptr = NULL;
  a->rowidx = NULL;
  a->val = NULL;
}

static void fill_values(synth_csc* a, uint64_t seed, uint64_t stream) {
  a->val = (float*)malloc(sizeof(float) * (size_t)(a->nnz > 0 ? a->nnz : 1));
  if (!a->val) return;
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < a->nnz; ++p) a->val[p] = draw_f32(seed, stream, (uint64_t)p);
}

static int cmp_i32(const void* x, const void* y) {
  int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
  return (a > b) - (a < b);
}

/*
 * Erdos-Renyi: every (i, j) present independently with probability p.
 * Column j walks geometric gaps (inverse CDF of the gap length), which
 * yields rows in ascending order.  Directed, self-loops allowed.
 * Row draws use stream 0 and counter (j << 32 | draw number); values use
 * `val_stream` and the entry position.
 */
int synth_erdos_renyi(int64_t m, int64_t n, double p, uint64_t seed, int want_val,
                      uint64_t val_stream, synth_csc* out) {
  memset(out, 0, sizeof(*out));
  if (m <= 0 || n <= 0 || m > INT32_MAX || n > INT32_MAX || !(p > 0.0) || !(p < 1.0)) return -1;
  out->m = m;
  out->n = n;
  int32_t* cnt = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
  if (!cnt) return -2;
  const double lq = log1p(-p);
  /* pass 1: count; pass 2: fill (same draws) */
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t j = 0; j < n; ++j) {
    int64_t r = -1, c = 0;
    for (uint64_t t = 0;; ++t) {
      double u = draw_f64_open0(seed, 0, ((uint64_t)j << 32) | t);
      double g = floor(log(u) / lq);
      if (g >= (double)m) break;
      r += (int64_t)g + 1;
      if (r >= m) break;
      ++c;
    }
    cnt[j + 1] = (int32_t)c;
  }
  out->colptr = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
  if (!out->colptr) { free(cnt); return -2; }
  out->colptr[0] = 0;
  for (int64_t j = 0; j < n; ++j) {
    int64_t nx = (int64_t)out->colptr[j] + cnt[j + 1];
    if (nx > INT32_MAX) { free(cnt); synth_free(out); return -3; }
    out->colptr[j + 1] = (int32_t)nx;
  }
  free(cnt);
  out->nnz = out->colptr[n];
  out->rowidx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(out->nnz > 0 ? out->nnz : 1));
  if (!out->rowidx) { synth_free(out); return -2; }
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t j = 0; j < n; ++j) {
    int64_t r = -1, q = out->colptr[j];
    for (uint64_t t = 0;; ++t) {
      double u = draw_f64_open0(seed, 0, ((uint64_t)j << 32) | t);
      double g = floor(log(u) / lq);
      if (g >= (double)m) break;
      r += (int64_t)g + 1;
      if (r >= m) break;
      out->rowidx[q++] = (int32_t)r;
    }
  }
  if (want_val) {
    fill_values(out, seed, val_stream);
    if (!out->val) { synth_free(out); return -2; }
  }
  return 0;
}

/*
 * R-MAT with quadrant probabilities (a, b, c, 1-a-b-c), no noise.
 * 2^scale vertices, edge_factor * 2^scale generated edges.  Edge e draws
 * one 64-bit word per two levels (stream 0, counter e * 32 + word).
 * Post-processing (a Graph500-style convention): symmetrise, drop
 * self-loops, merge duplicates, and if `permute` relabel vertices by a
 * seeded Fisher-Yates permutation (stream 1).  Rows ascend in each column.
 */
int synth_rmat(int scale, int64_t edge_factor, double a, double b, double c, uint64_t seed,
               int permute, int want_val, uint64_t val_stream, synth_csc* out) {
  memset(out, 0, sizeof(*out));
  if (scale < 1 || scale > 30 || edge_factor < 1) return -1;
  const int64_t n = (int64_t)1 << scale;
  const int64_t ne = edge_factor * n;
  if (2 * ne > INT32_MAX) return -3;
  out->m = n;
  out->n = n;
  /* integer thresholds on 32-bit draws */
  const uint64_t ta = (uint64_t)(a * 4294967296.0);
  const uint64_t tab = (uint64_t)((a + b) * 4294967296.0);
  const uint64_t tabc = (uint64_t)((a + b + c) * 4294967296.0);

  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* src = (int32_t*)malloc(sizeof(int32_t) * (size_t)ne);
  int32_t* dst = (int32_t*)malloc(sizeof(int32_t) * (size_t)ne);
  int32_t* cnt = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
  if (!perm || !src || !dst || !cnt) { free(perm); free(src); free(dst); free(cnt); return -2; }
  for (int64_t v = 0; v < n; ++v) perm[v] = (int32_t)v;
  if (permute) {
    for (int64_t i = n - 1; i > 0; --i) {
      uint64_t r = draw(seed, 1, (uint64_t)i);
      int64_t j = (int64_t)(((unsigned __int128)r * (uint64_t)(i + 1)) >> 64);
      int32_t t = perm[i];
      perm[i] = perm[j];
      perm[j] = t;
    }
  }
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < ne; ++e) {
    uint64_t u = 0, v = 0, w = 0;
    for (int l = 0; l < scale; ++l) {
      if ((l & 1) == 0) w = draw(seed, 0, (uint64_t)e * 32 + (uint64_t)(l >> 1));
      uint64_t r = (l & 1) ? (w >> 32) : (w & 0xFFFFFFFFULL);
      uint64_t bu, bv;
      if (r < ta) { bu = 0; bv = 0; }
      else if (r < tab) { bu = 0; bv = 1; }
      else if (r < tabc) { bu = 1; bv = 0; }
      else { bu = 1; bv = 1; }
      u = (u << 1) | bu;
      v = (v << 1) | bv;
    }
    src[e] = perm[u];
    dst[e] = perm[v];
  }
  free(perm);
  /* count both directions per column, self-loops dropped */
  for (int64_t e = 0; e < ne; ++e) {
    if (src[e] == dst[e]) continue;
    cnt[src[e] + 1]++;
    cnt[dst[e] + 1]++;
  }
  int64_t* start = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  if (!start) { free(src); free(dst); free(cnt); return -2; }
  start[0] = 0;
  for (int64_t v = 0; v < n; ++v) start[v + 1] = start[v] + cnt[v + 1];
  int64_t tot = start[n];
  int32_t* rows = (int32_t*)malloc(sizeof(int32_t) * (size_t)(tot > 0 ? tot : 1));
  int64_t* fillp = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!rows || !fillp) { free(src); free(dst); free(cnt); free(start); free(rows); free(fillp); return -2; }
  for (int64_t v = 0; v < n; ++v) fillp[v] = start[v];
  /* column src gets row dst and column dst gets row src */
  for (int64_t e = 0; e < ne; ++e) {
    int32_t s = src[e], d = dst[e];
    if (s == d) continue;
    rows[fillp[s]++] = d;
    rows[fillp[d]++] = s;
  }
  free(src);
  free(dst);
  free(fillp);
  /* sort and merge duplicates per column */
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t v = 0; v < n; ++v) {
    int64_t b0 = start[v], e0 = start[v + 1];
    if (e0 - b0 > 1) qsort(rows + b0, (size_t)(e0 - b0), sizeof(int32_t), cmp_i32);
    int64_t q = b0;
    for (int64_t p = b0; p < e0; ++p)
      if (p == b0 || rows[p] != rows[p - 1]) rows[q++] = rows[p];
    cnt[v + 1] = (int32_t)(q - b0);
  }
  out->colptr = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
  if (!out->colptr) { free(cnt); free(start); free(rows); return -2; }
  out->colptr[0] = 0;
  for (int64_t v = 0; v < n; ++v) out->colptr[v + 1] = out->colptr[v] + cnt[v + 1];
  out->nnz = out->colptr[n];
  out->rowidx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(out->nnz > 0 ? out->nnz : 1));
  if (!out->rowidx) { free(cnt); free(start); free(rows); synth_free(out); return -2; }
#pragma omp parallel for schedule(static)
  for (int64_t v = 0; v < n; ++v)
    memcpy(out->rowidx + out->colptr[v], rows + start[v], sizeof(int32_t) * (size_t)cnt[v + 1]);
  free(cnt);
  free(start);
  free(rows);
  if (want_val) {
    fill_values(out, seed, val_stream);
    if (!out->val) { synth_free(out); return -2; }
  }
  return 0;
}

/*
 * X-by-Y-by-Z grid (Z=1 gives a 2D 5-point grid), vertex id
 * x*Y*Z + y*Z + z, an entry for every present grid neighbour (no
 * diagonal).  Undirected edge (v, v + step along axis d) is identified by
 * 3*v + d and removed, in both directions, when its draw (stream 0)
 * falls below remove_frac.  Rows ascend in each column.
 */
static inline int grid_edge_kept(uint64_t seed, uint64_t thr, int64_t v, int d) {
  if (thr == 0) return 1;
  return (draw(seed, 0, (uint64_t)(3 * v + d)) >> 32) >= thr;
}

int synth_grid3d(int64_t X, int64_t Y, int64_t Z, double remove_frac, uint64_t seed,
                 int want_val, uint64_t val_stream, synth_csc* out) {
  memset(out, 0, sizeof(*out));
  if (X < 1 || Y < 1 || Z < 1 || remove_frac < 0.0 || remove_frac >= 1.0) return -1;
  const int64_t n = X * Y * Z;
  if (n > INT32_MAX || 6 * n > INT32_MAX) return -3;
  const uint64_t thr = (uint64_t)(remove_frac * 4294967296.0);
  const int64_t sx = Y * Z, sy = Z;
  out->m = n;
  out->n = n;
  out->colptr = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
  if (!out->colptr) return -2;
  out->colptr[0] = 0;
  /* neighbours in ascending id order: -x, -y, -z, +z, +y, +x */
#define GRID_NEIGHBOURS(BODY)                                                     \
  {                                                                              \
    int64_t x = v / sx, y = (v / sy) % Y, z = v % Z;                             \
    if (x > 0 && grid_edge_kept(seed, thr, v - sx, 0)) { int64_t u = v - sx; BODY } \
    if (y > 0 && grid_edge_kept(seed, thr, v - sy, 1)) { int64_t u = v - sy; BODY } \
    if (z > 0 && grid_edge_kept(seed, thr, v - 1, 2)) { int64_t u = v - 1; BODY }   \
    if (z + 1 < Z && grid_edge_kept(seed, thr, v, 2)) { int64_t u = v + 1; BODY }   \
    if (y + 1 < Y && grid_edge_kept(seed, thr, v, 1)) { int64_t u = v + sy; BODY }  \
    if (x + 1 < X && grid_edge_kept(seed, thr, v, 0)) { int64_t u = v + sx; BODY }  \
  }
#pragma omp parallel for schedule(static)
  for (int64_t v = 0; v < n; ++v) {
    int32_t c = 0;
    GRID_NEIGHBOURS({ (void)u; ++c; })
    out->colptr[v + 1] = c;
  }
  for (int64_t v = 0; v < n; ++v) out->colptr[v + 1] += out->colptr[v];
  out->nnz = out->colptr[n];
  out->rowidx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(out->nnz > 0 ? out->nnz : 1));
  if (!out->rowidx) { synth_free(out); return -2; }
#pragma omp parallel for schedule(static)
  for (int64_t v = 0; v < n; ++v) {
    int64_t q = out->colptr[v];
    GRID_NEIGHBOURS({ out->rowidx[q++] = (int32_t)u; })
  }
#undef GRID_NEIGHBOURS
  if (want_val) {
    fill_values(out, seed, val_stream);
    if (!out->val) { synth_free(out); return -2; }
  }
  return 0;
}

/* Uniform float values in [0,1) for k draws of (seed, stream). */
void synth_uniform_f32(uint64_t seed, uint64_t stream, int64_t k, float* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < k; ++i) out[i] = draw_f32(seed, stream, (uint64_t)i);
}

/*
 * f distinct indices uniform in [0, n): the first f entries of a seeded
 * Fisher-Yates shuffle (stream `stream`), in shuffle order (unsorted).
 * scratch must hold n int32.
 */
int synth_sample_distinct(int64_t n, int64_t f, uint64_t seed, uint64_t stream,
                          int32_t* scratch, int32_t* out) {
  if (n < 0 || f < 0 || f > n || n > INT32_MAX) return -1;
  for (int64_t i = 0; i < n; ++i) scratch[i] = (int32_t)i;
  for (int64_t i = 0; i < f; ++i) {
    uint64_t r = draw(seed, stream, (uint64_t)i);
    int64_t j = i + (int64_t)(((unsigned __int128)r * (uint64_t)(n - i)) >> 64);
    int32_t t = scratch[i];
    scratch[i] = scratch[j];
    scratch[j] = t;
    out[i] = scratch[i];
  }
  return 0;
}

/* Number of threads the generators run on (1 without OpenMP). */
int synth_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
