/*
 * Sequential CPU oracle for sparse-matrix x sparse-vector products (SpMSpV)
 * over a semiring, and for the breadth-first search built from them.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously
 * correct statement of what the GPU path computes.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * GPU library never calls it and shares no code, header or constant with it.
 *
 * Paper: Azad & Buluc, "A work-efficient parallel sparse matrix-sparse
 * vector multiplication algorithm" (arXiv 1610.07902).
 *
 *  - Problem statement y <- A x, A m-by-n in CSC, x and y sparse lists:
 *    Sec. II-A (Notation) and Sec. II-C (data structures).
 *  - Method: the sequential Gustavson-style column walk into a sparse
 *    accumulator (SPA) named in Sec. I, with the SPA initialised only where
 *    it is touched (Sec. II-F, second requirement).  The bucketed parallel
 *    algorithm (Algorithm 1) computes exactly this result; only the order
 *    of the additions differs.
 *  - The multiply count equals the sum of the selected column lengths,
 *    the Omega(df) lower bound of Sec. II-D.
 *
 * Readings of points the paper leaves open (each is also listed with the
 * design notes of the project):
 *  - Operand order is A(i,j) (x) x(j) (the GraphBLAS mxv order).  With
 *    this order select2nd returns x(j), which is what BFS needs.
 *  - The index set of y is structural: a row that receives at least one
 *    product is present even when its sum is exactly zero (Algorithm 1,
 *    Step 2, records every touched index in uind_k).
 *  - A separate "touched" flag replaces the infinity sentinel of
 *    Algorithm 1 so that any value, including INT32_MAX, is legal.
 *  - Mask (GraphBLAS style, future work in Sec. V): with complement=1 a
 *    row i may appear in y only where mask[i]==0; with complement=0 only
 *    where mask[i]!=0.  The multiply count includes masked products
 *    because every selected column entry is still read.
 *  - Floating point: float inputs are widened to double and accumulated
 *    in double; the integer semiring accumulates in int32.
 *  - Output y is returned sorted by index (the sorted-list format of
 *    Sec. II-C); unsorted-mode comparisons sort the other side.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PLUS_TIMES 0     /* (+, *)            over double            */
#define ORC_MIN_SELECT2ND 1  /* (min, select2nd)  over int32            */
#define ORC_OR_AND 2         /* (or, and)         over {0,1}            */

#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_DUPLICATE_X -2
#define ORC_ERR_NOMEM -3

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* Workspace of one dense SPA of length m: values, touched flags and the
 * list of touched indices (Sec. II-E describes the SPA as a dense value
 * vector plus a list of the indices it holds). */
typedef struct {
  int32_t m;
  double* vd;       /* values for (+,*)           */
  int32_t* vi;      /* values for (min,select2nd) */
  uint8_t* touched; /* 1 where the SPA holds a value */
  int32_t* list;    /* touched indices, in first-touch order */
  uint8_t* xseen;   /* n flags to reject duplicate x indices */
  int32_t n;
} orc_spa;

static int spa_init(orc_spa* s, int32_t m, int32_t n) {
  s->m = m;
  s->n = n;
  s->vd = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  s->vi = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  s->touched = (uint8_t*)calloc((size_t)(m > 0 ? m : 1), 1);
  s->list = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  s->xseen = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  if (!s->vd || !s->vi || !s->touched || !s->list || !s->xseen) return ORC_ERR_NOMEM;
  return ORC_OK;
}

static void spa_free(orc_spa* s) {
  free(s->vd);
  free(s->vi);
  free(s->touched);
  free(s->list);
  free(s->xseen);
}

/* One SpMSpV through an already allocated SPA.  The SPA's touched flags
 * are all zero on entry and are reset (only where set) before return. */
static int64_t spmspv_core(orc_spa* s, int semiring, const int32_t* colptr,
                           const int32_t* rowidx, const float* val,
                           const int32_t* x_idx, const void* x_val, int32_t f,
                           const uint8_t* mask, int complement,
                           int32_t* y_idx, void* y_val, int32_t* nnz_y,
                           double* y_absum, int* err) {
  int64_t nmult = 0;
  int32_t nt = 0;
  *err = ORC_OK;
  /* duplicate check: the list format holds one entry per index (Sec. II-C) */
  for (int32_t k = 0; k < f; ++k) {
    int32_t j = x_idx[k];
    if (j < 0 || j >= s->n) { *err = ORC_ERR_ARG; break; }
    if (s->xseen[j]) { *err = ORC_ERR_DUPLICATE_X; break; }
    s->xseen[j] = 1;
  }
  for (int32_t k = 0; k < f; ++k) {
    int32_t j = x_idx[k];
    if (j >= 0 && j < s->n) s->xseen[j] = 0;
  }
  if (*err != ORC_OK) { *nnz_y = 0; return 0; }

  /* Gustavson column walk: for every x(j) present, for every A(i,j) present */
  for (int32_t k = 0; k < f; ++k) {
    int32_t j = x_idx[k];
    for (int32_t p = colptr[j]; p < colptr[j + 1]; ++p) {
      int32_t i = rowidx[p];
      ++nmult; /* every selected column entry is one multiplication */
      if (mask) {
        int in_mask = mask[i] != 0;
        if (complement ? in_mask : !in_mask) continue;
      }
      if (semiring == ORC_PLUS_TIMES) {
        double a = val ? (double)val[p] : 1.0;
        double xv = (double)((const float*)x_val)[k];
        double t = a * xv;
        if (!s->touched[i]) {
          s->touched[i] = 1;
          s->list[nt++] = i;
          s->vd[i] = t;
        } else {
          s->vd[i] += t;
        }
      } else if (semiring == ORC_MIN_SELECT2ND) {
        int32_t t = ((const int32_t*)x_val)[k]; /* select2nd(A(i,j), x(j)) = x(j) */
        if (!s->touched[i]) {
          s->touched[i] = 1;
          s->list[nt++] = i;
          s->vi[i] = t;
        } else if (t < s->vi[i]) {
          s->vi[i] = t;
        }
      } else { /* ORC_OR_AND: every present x(j) and A(i,j) is true */
        if (!s->touched[i]) {
          s->touched[i] = 1;
          s->list[nt++] = i;
        }
      }
    }
  }

  /* sum of |a*x| per output row, the scale of the floating-point bound */
  if (y_absum && semiring == ORC_PLUS_TIMES) {
    for (int32_t q = 0; q < nt; ++q) s->vi[s->list[q]] = q;
    for (int32_t q = 0; q < nt; ++q) y_absum[q] = 0.0;
    for (int32_t k = 0; k < f; ++k) {
      int32_t j = x_idx[k];
      for (int32_t p = colptr[j]; p < colptr[j + 1]; ++p) {
        int32_t i = rowidx[p];
        if (!s->touched[i]) continue;
        double a = val ? (double)val[p] : 1.0;
        double t = a * (double)((const float*)x_val)[k];
        y_absum[s->vi[i]] += t < 0 ? -t : t;
      }
    }
  }

  /* output in sorted-list format */
  qsort(s->list, (size_t)nt, sizeof(int32_t), cmp_i32);
  if (y_absum && semiring == ORC_PLUS_TIMES) {
    /* reorder the absolute sums to the sorted order */
    double* tmp = (double*)malloc(sizeof(double) * (size_t)(nt > 0 ? nt : 1));
    for (int32_t q = 0; q < nt; ++q) tmp[q] = y_absum[s->vi[s->list[q]]];
    memcpy(y_absum, tmp, sizeof(double) * (size_t)nt);
    free(tmp);
  }
  for (int32_t q = 0; q < nt; ++q) {
    int32_t i = s->list[q];
    if (y_idx) y_idx[q] = i;
    if (y_val) {
      if (semiring == ORC_PLUS_TIMES) ((double*)y_val)[q] = s->vd[i];
      else if (semiring == ORC_MIN_SELECT2ND) ((int32_t*)y_val)[q] = s->vi[i];
    }
    s->touched[i] = 0; /* partial reset: only what was touched (Sec. II-F) */
  }
  *nnz_y = nt;
  return nmult;
}

/*
 * y <- A (+).(x) x.  x_val is float[f] for (+,*) (NULL allowed for all-ones
 * is NOT accepted: pass the values), int32[f] for (min,select2nd), ignored
 * for (or,and).  y_idx must hold min(m, sum of selected column lengths)
 * entries.  y_val receives double[] for (+,*), int32[] for (min,select2nd)
 * and may be NULL.  y_absum (may be NULL) receives sum_j |A(i,j) x(j)| per
 * output row, for (+,*) only.  Returns the multiply count (>= 0) or a
 * negative ORC_ERR_* code.
 */
int64_t oracle_spmspv(int32_t m, int32_t n, const int32_t* colptr,
                      const int32_t* rowidx, const float* val, int semiring,
                      const int32_t* x_idx, const void* x_val, int32_t f,
                      const uint8_t* mask, int complement, int32_t* y_idx,
                      void* y_val, double* y_absum, int32_t* nnz_y) {
  if (m < 0 || n < 0 || f < 0 || !colptr || (f > 0 && !x_idx)) return ORC_ERR_ARG;
  if (semiring < 0 || semiring > 2) return ORC_ERR_ARG;
  if (semiring != ORC_OR_AND && f > 0 && !x_val) return ORC_ERR_ARG;
  orc_spa s;
  if (spa_init(&s, m, n) != ORC_OK) { spa_free(&s); return ORC_ERR_NOMEM; }
  int err = ORC_OK;
  int64_t nmult = spmspv_core(&s, semiring, colptr, rowidx, val, x_idx, x_val, f,
                              mask, complement, y_idx, y_val, nnz_y, y_absum, &err);
  spa_free(&s);
  return err != ORC_OK ? (int64_t)err : nmult;
}

/*
 * Breadth-first search as repeated masked (min, select2nd) SpMSpV
 * (Sec. IV-D uses BFS as the customer of SpMSpV; the product of the
 * adjacency matrix with the frontier gives the next frontier).
 * Reading of the level rule: level[src]=0 and parent[src]=src; frontier
 * x_0 = {(src, src)}; visited = {src}.  At step L, y = A (min.select2nd) x
 * restricted to unvisited rows; every (i, p) in y gets level L, parent p
 * (the smallest-id frontier neighbour), joins visited, and the next
 * frontier is {(i, i)}.  Stop when y is empty.  Unreached: level = parent = -1.
 * A must be square; for an undirected graph it is symmetric.
 * Returns the number of levels (max level + 1), or a negative error.
 * total_mult (may be NULL) receives the summed multiply count.
 * level_sizes (may be NULL, n entries) receives the frontier size per level.
 */
int32_t oracle_bfs(int32_t n, const int32_t* colptr, const int32_t* rowidx,
                   int32_t src, int32_t* level, int32_t* parent,
                   int64_t* total_mult, int32_t* level_sizes) {
  if (n <= 0 || src < 0 || src >= n || !colptr || !level || !parent) return ORC_ERR_ARG;
  orc_spa s;
  if (spa_init(&s, n, n) != ORC_OK) { spa_free(&s); return ORC_ERR_NOMEM; }
  uint8_t* visited = (uint8_t*)calloc((size_t)n, 1);
  int32_t* xi = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* xv = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* yi = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* yv = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!visited || !xi || !xv || !yi || !yv) {
    spa_free(&s); free(visited); free(xi); free(xv); free(yi); free(yv);
    return ORC_ERR_NOMEM;
  }
  for (int32_t i = 0; i < n; ++i) { level[i] = -1; parent[i] = -1; }
  level[src] = 0;
  parent[src] = src;
  visited[src] = 1;
  xi[0] = src;
  xv[0] = src;
  int32_t f = 1, L = 0;
  int64_t tm = 0;
  if (level_sizes) level_sizes[0] = 1;
  for (;;) {
    int32_t ny = 0;
    int err = ORC_OK;
    tm += spmspv_core(&s, ORC_MIN_SELECT2ND, colptr, rowidx, NULL, xi, xv, f, visited,
                      1, yi, yv, &ny, NULL, &err);
    if (err != ORC_OK) { L = err; break; }
    if (ny == 0) break;
    ++L;
    for (int32_t q = 0; q < ny; ++q) {
      int32_t i = yi[q];
      level[i] = L;
      parent[i] = yv[q];
      visited[i] = 1;
      xi[q] = i;
      xv[q] = i;
    }
    if (level_sizes) level_sizes[L] = ny;
    f = ny;
  }
  spa_free(&s);
  free(visited); free(xi); free(xv); free(yi); free(yv);
  if (total_mult) *total_mult = tm;
  return L < 0 ? L : L + 1;
}

/*
 * The same breadth-first search, but each level's product is computed by
 * the matrix-driven (pull) definition: for every unvisited row i,
 * y(i) = min { j : A(i,j) present, j in the frontier }.  Matrix-driven
 * SpMSpV is the class of Sec. II-B; "pull" and "push" give one result.
 * It reads A by rows, so A must be symmetric (CSC read as CSR).
 * Returns the number of levels.
 */
int32_t oracle_bfs_pull(int32_t n, const int32_t* colptr, const int32_t* rowidx,
                        int32_t src, int32_t* level, int32_t* parent) {
  if (n <= 0 || src < 0 || src >= n || !colptr || !level || !parent) return ORC_ERR_ARG;
  uint8_t* front = (uint8_t*)calloc((size_t)n, 1);
  uint8_t* next = (uint8_t*)calloc((size_t)n, 1);
  if (!front || !next) { free(front); free(next); return ORC_ERR_NOMEM; }
  for (int32_t i = 0; i < n; ++i) { level[i] = -1; parent[i] = -1; }
  level[src] = 0;
  parent[src] = src;
  front[src] = 1;
  int32_t L = 0;
  for (;;) {
    int32_t found = 0;
    for (int32_t i = 0; i < n; ++i) {
      next[i] = 0;
      if (level[i] >= 0) continue;
      int32_t best = -1;
      for (int32_t p = colptr[i]; p < colptr[i + 1]; ++p) {
        int32_t j = rowidx[p];
        if (front[j] && (best < 0 || j < best)) best = j;
      }
      if (best >= 0) { parent[i] = best; next[i] = 1; ++found; }
    }
    if (!found) break;
    ++L;
    for (int32_t i = 0; i < n; ++i) {
      if (next[i]) level[i] = L;
      front[i] = next[i];
    }
  }
  free(front);
  free(next);
  return L + 1;
}

/*
 * Connected components of an undirected graph given as a pattern-symmetric
 * CSC matrix (Sec. I names connected components among the SpMSpV-built graph
 * algorithms).  The result has a plain definition: label[v] is the smallest
 * vertex id in the component of v.  Written as that definition: union-find
 * over every stored edge (i, j), then each vertex takes the smallest id found
 * in its set.  Returns the number of components, or -1 on a bad row id.
 */
static int32_t uf_find(int32_t* up, int32_t v) {
  while (up[v] != v) {
    up[v] = up[up[v]];  /* path halving */
    v = up[v];
  }
  return v;
}

int32_t oracle_cc(int32_t n, const int32_t* colptr, const int32_t* rowidx, int32_t* label) {
  int32_t* up = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t* low = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (!up || !low) {
    free(up);
    free(low);
    return -2;
  }
  for (int32_t v = 0; v < n; ++v) up[v] = v;
  for (int32_t j = 0; j < n; ++j) {
    for (int32_t p = colptr[j]; p < colptr[j + 1]; ++p) {
      const int32_t i = rowidx[p];
      if (i < 0 || i >= n) {
        free(up);
        free(low);
        return -1;
      }
      const int32_t a = uf_find(up, i), b = uf_find(up, j);
      if (a != b) up[a] = b;
    }
  }
  for (int32_t v = 0; v < n; ++v) low[v] = n;
  int32_t comps = 0;
  for (int32_t v = 0; v < n; ++v) {
    const int32_t r = uf_find(up, v);
    if (low[r] == n) ++comps;
    if (v < low[r]) low[r] = v;
  }
  for (int32_t v = 0; v < n; ++v) label[v] = low[uf_find(up, v)];
  free(up);
  free(low);
  return comps;
}

/*
 * Maximal independent set of an undirected graph (pattern-symmetric CSC),
 * the set Luby's rounds reach with fixed, distinct priorities (Sec. I names
 * maximal independent sets among the SpMSpV-built graph algorithms).  That
 * set has a plain definition, written out here: take the vertices in order
 * of increasing priority and keep each one none of whose neighbours has been
 * kept (the greedy set in priority order).  in_set[v] = 1 if kept, else 0.
 * Returns the size of the set, -1 on a bad row id, -3 if priorities repeat.
 */
static const int32_t* g_prio_for_sort;
static int cmp_by_prio(const void* a, const void* b) {
  const int32_t pa = g_prio_for_sort[*(const int32_t*)a], pb = g_prio_for_sort[*(const int32_t*)b];
  return (pa > pb) - (pa < pb);
}

int32_t oracle_mis(int32_t n, const int32_t* colptr, const int32_t* rowidx, const int32_t* prio,
                   int32_t* in_set) {
  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (!order) return -2;
  for (int32_t v = 0; v < n; ++v) {
    order[v] = v;
    in_set[v] = 0;
  }
  g_prio_for_sort = prio;
  qsort(order, (size_t)n, sizeof(int32_t), cmp_by_prio);
  for (int32_t k = 1; k < n; ++k)
    if (prio[order[k]] == prio[order[k - 1]]) {
      free(order);
      return -3;
    }
  int32_t size = 0;
  for (int32_t k = 0; k < n; ++k) {
    const int32_t v = order[k];
    int keep = 1;
    for (int32_t p = colptr[v]; p < colptr[v + 1]; ++p) {
      const int32_t u = rowidx[p];
      if (u < 0 || u >= n) {
        free(order);
        return -1;
      }
      if (u != v && in_set[u]) {
        keep = 0;
        break;
      }
    }
    if (keep) {
      in_set[v] = 1;
      ++size;
    }
  }
  free(order);
  return size;
}

/*
 * Maximum-cardinality matching of the bipartite graph whose two sides are the
 * rows and the columns of A (m-by-n CSC; an edge joins row i and column j when
 * A(i,j) is stored).  Sec. I names bipartite graph matching among the
 * SpMSpV-built graph algorithms.  The cardinality has a plain definition, the
 * largest number of edges no two of which share an end; the matching itself
 * is one of possibly many.  Method: augmenting paths (Berge: a matching is
 * maximum exactly when no augmenting path is left), searched depth first
 * from each column in turn, with the rows seen in this search stamped so that
 * each is tried once (Kuhn's algorithm, written with an explicit stack).
 * mate_r[i] = matched column of row i or -1; mate_c[j] = matched row or -1.
 * Returns the cardinality, -1 on a bad row id, -2 out of memory.
 */
int32_t oracle_mcm(int32_t m, int32_t n, const int32_t* colptr, const int32_t* rowidx,
                   int32_t* mate_r, int32_t* mate_c) {
  int32_t* stamp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  int32_t* scol = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  int32_t* spos = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  if (!stamp || !scol || !spos) {
    free(stamp);
    free(scol);
    free(spos);
    return -2;
  }
  for (int32_t i = 0; i < m; ++i) {
    mate_r[i] = -1;
    stamp[i] = -1;
  }
  for (int32_t j = 0; j < n; ++j) mate_c[j] = -1;
  int32_t size = 0;
  for (int32_t r = 0; r < n; ++r) {
    int32_t depth = 0, found = -1;
    scol[0] = r;
    spos[0] = colptr[r];
    while (depth >= 0) {
      const int32_t j = scol[depth];
      const int32_t p = spos[depth];
      if (p == colptr[j + 1]) {  /* every row of column j tried: back up */
        --depth;
        continue;
      }
      spos[depth] = p + 1;
      const int32_t i = rowidx[p];
      if (i < 0 || i >= m) {
        free(stamp);
        free(scol);
        free(spos);
        return -1;
      }
      if (stamp[i] == r) continue;
      stamp[i] = r;
      if (mate_r[i] < 0) {  /* a free row ends an augmenting path */
        found = i;
        break;
      }
      ++depth;  /* continue the alternating path through the column matched to row i */
      scol[depth] = mate_r[i];
      spos[depth] = colptr[mate_r[i]];
    }
    if (found < 0) continue;
    /* flip the path: the column at each depth takes the row reached from it,
       giving up the row it was entered through (its old mate) to the column below */
    int32_t i = found;
    for (int32_t d = depth; d >= 0; --d) {
      const int32_t j = scol[d];
      const int32_t old = mate_c[j];
      mate_c[j] = i;
      mate_r[i] = j;
      i = old;
    }
    ++size;
  }
  free(stamp);
  free(scol);
  free(spos);
  return size;
}
