/*
 * spmspv.h - C ABI of the GB300 (sm_103a) sparse-matrix x sparse-vector
 * library: y <- A (+).(x) x over a semiring, A in CSC form, x and y in list
 * (index, value) form.
 *
 * Paper: A. Azad, A. Buluc, "A work-efficient parallel sparse matrix-sparse
 * vector multiplication algorithm", arXiv 1610.07902.
 *   Operation and notation ........ Sec. II-A
 *   CSC matrix, list-format vectors, output format = input format ... Sec. II-C
 *   The bucketed algorithm ......... Sec. III, Algorithm 1 (Steps 1-3), Algorithm 2
 *   Preallocated buckets and SPA ... Sec. III-A ("Memory allocation")
 *   Masked SpMSpV .................. Sec. V (GraphBLAS masks, future work there)
 *   BFS as repeated SpMSpV ......... Sec. IV-D
 *
 * Conventions shared by every call:
 *   - Every function returns an int status: SPMSPV_OK (0) or an SPMSPV_ERR_*
 *     code.  spmspv_last_error() gives a message owned by the library.
 *   - Every array argument is a DEVICE pointer owned by the caller unless the
 *     argument's comment says "host".
 *   - A handle BORROWS the CSC arrays given at create: they must stay
 *     allocated and unchanged until spmspv_destroy.  The handle OWNS its
 *     workspace (buckets, compacted frontier, scan state), allocated once at
 *     create, as the paper preallocates buckets and the SPA once (Sec. III-A).
 *   - Calls that take a stream are asynchronous on that stream and make no
 *     host synchronisation.  A handle runs one product at a time: calls on a
 *     handle must be ordered (same stream, or externally synchronised).
 *   - Errors found on the device (output capacity exceeded, a wait that ran
 *     out) are recorded in a device status word; spmspv_device_status()
 *     synchronises the handle's last stream and returns and clears it.
 *   - Index type int32, floating values float32.  nnz(A) < 2^31.
 */
#ifndef SPMSPV_H_
#define SPMSPV_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t without the CUDA headers; NULL is the legacy default stream */
typedef struct CUstream_st* spmspv_stream_t;
typedef struct spmspv_handle spmspv_handle;

/* ---- status codes ---- */
#define SPMSPV_OK 0
#define SPMSPV_ERR_ARG 1         /* invalid argument (null pointer, size, id) */
#define SPMSPV_ERR_STATE 2       /* handle not usable (destroyed, wrong device) */
#define SPMSPV_ERR_OOM 3         /* device allocation failed at create */
#define SPMSPV_ERR_CUDA 4        /* a CUDA runtime call failed */
#define SPMSPV_ERR_CAPACITY 5    /* y needs more entries than y_capacity */
#define SPMSPV_ERR_TIMEOUT 6     /* a bounded device-side wait gave up */
#define SPMSPV_ERR_INDEX 7       /* index out of range (checked inputs) */
#define SPMSPV_ERR_UNSUPPORTED 8 /* shape or option outside the supported range */

/* ---- matrix value types (spmspv_create_csc val_type) ---- */
#define SPMSPV_VAL_NONE 0 /* pattern matrix: every stored A(i,j) is 1 */
#define SPMSPV_VAL_F32 1  /* float values */

/* ---- create flags ---- */
#define SPMSPV_CSC_PATTERN_SYMMETRIC 1u /* A and A^T have the same nonzero pattern: the CSC
                                           doubles as CSR for the pull direction of the
                                           (min,select2nd) and (or,and) semirings */
#define SPMSPV_CSC_SYMMETRIC 3u         /* A == A^T, values included: pull also for (+,*) */

/* ---- semirings (spmspv_run semiring) ----
 * Operand order A(i,j) (x) x(j), the GraphBLAS mxv order.
 *   PLUS_TIMES_F32   : (x) = a*x, (+) = +, float32.  x_val, y_val: float[].
 *                      y's index set is structural (a sum that is exactly 0
 *                      still appears).
 *   MIN_SELECT2ND_I32: (x) = x(j) (select2nd), (+) = min, int32.
 *                      x_val, y_val: int32[].  Matrix values are not read.
 *   OR_AND_BOOL      : (x) = and, (+) = or.  Values are implicit true:
 *                      x_val and y_val are ignored (may be NULL); y is the
 *                      index set only.                                       */
#define SPMSPV_PLUS_TIMES_F32 0
#define SPMSPV_MIN_SELECT2ND_I32 1
#define SPMSPV_OR_AND_BOOL 2

/* ---- run options (spmspv_run opts) ---- */
#define SPMSPV_MASK_COMPLEMENT 1u /* keep row i only where mask bit i is 0 */
#define SPMSPV_SORTED_OUT 2u      /* y_idx ascending (see note below) */
#define SPMSPV_SCHED_AUTO 4u      /* let the learned selector pick the schedule (a call
                                     without a mask stays push) */
#define SPMSPV_SCHED_FORCE 8u     /* use schedule SPMSPV_SCHED_ID(opts) */
#define SPMSPV_WITH_FEATURES 16u  /* also compute the selector features (spmspv_last_features)
                                     with a fixed schedule; costs a pass over the mask */
#define SPMSPV_SORT_X 32u         /* sort x by index on the device first (Sec. III-A, cache
                                     efficiency: more local column accesses for denser x);
                                     a counting sort over [0, n), about n/8 + 12 nnz(x)
                                     bytes of traffic; buffers of 16n bytes on first use */
#define SPMSPV_BUCKETS_ONLY 128u   /* spmspv_run, (+,*): never the direct form (see below) */
#define SPMSPV_SCHED_RULE 64u       /* spmspv_bfs only: push or pull per level by the
                                       direction-optimizing rule of Beamer, Asanovic and
                                       Patterson (SC 2012; two fixed thresholds, alpha = 14,
                                       beta = 24), the baseline of the learned selector */
#define SPMSPV_X_IDS 65536u          /* (min, select2nd): the caller states that every x value
                                       equals its index (a BFS frontier); the pull direction
                                       then stops at a row's first frontier neighbour when row
                                       ids ascend in every column (the first is the smallest),
                                       as the BFS loop does.  Other x values give undefined y */
#define SPMSPV_SCHED_SHIFT 8
#define SPMSPV_SCHED_OPT(s) (SPMSPV_SCHED_FORCE | ((uint32_t)(s) << SPMSPV_SCHED_SHIFT))
#define SPMSPV_SCHED_ID(opts) (((opts) >> SPMSPV_SCHED_SHIFT) & 0xFFu)
#define SPMSPV_NUM_SCHEDULES 12

/* ---- device status bits (spmspv_device_status) ---- */
#define SPMSPV_DEV_CAPACITY 1u /* y did not fit; *d_nnz_y holds the size needed */
#define SPMSPV_DEV_TIMEOUT 2u  /* a bounded wait gave up; outputs are invalid */
#define SPMSPV_DEV_INDEX 4u    /* an x index was outside [0, n), or a bucket overflowed
                                  (duplicate x indices); outputs are invalid */
#define SPMSPV_DEV_BOUND 8u    /* a device loop reached the iteration bound its
                                  mathematics guarantees (matching); outputs are invalid */

/* Message for the last error returned on this thread (library-owned). */
const char* spmspv_last_error(void);

/*
 * Create a handle over an m-by-n CSC matrix (Sec. II-C: colptrs n+1,
 * rowids nnz, values nnz; row ids inside a column need not be sorted).
 *   h        host out: the new handle.
 *   m, n     rows, columns; 1 <= m <= 2^26, 1 <= n < 2^31.
 *   nnz      colptr[n]; 0 <= nnz < 2^31.
 *   colptr   device int32[n+1], non-decreasing, colptr[0] = 0.
 *   rowidx   device int32[nnz], each in [0, m).
 *   val      device float[nnz] for SPMSPV_VAL_F32, ignored (may be NULL)
 *            for SPMSPV_VAL_NONE.
 *   flags    SPMSPV_CSC_PATTERN_SYMMETRIC, SPMSPV_CSC_SYMMETRIC or 0.  The
 *            flags are trusted, not checked.
 * Synchronous: allocates the workspace (about 6 bytes per nonzero for the
 * buckets plus 16 bytes per column, and 4 bytes per row for the direct
 * form's accumulator when m <= 2^24) on the current device, and scans
 * rowidx once to size the row-range buckets.  Errors: ARG, OOM, CUDA,
 * UNSUPPORTED (m too large for the bucket row width).
 * A handle's calls use its one workspace: calls on the same handle must not
 * run at the same time on the GPU (issue them on one stream, or order the
 * streams); different handles are independent.
 */
int spmspv_create_csc(spmspv_handle** h, int32_t m, int32_t n, int64_t nnz,
                      const int32_t* colptr, const int32_t* rowidx, const void* val,
                      int val_type, uint32_t flags);

/*
 * Same, for a matrix in DCSC (Sec. II-C): only the nzc columns that hold an
 * entry are stored.  jc: device int32[nzc], their column ids, strictly
 * ascending in [0, n); cp: device int32[nzc+1], cp[0] = 0, non-decreasing,
 * cp[nzc] = nnz, the entries of stored column p being rowidx/val[cp[p] ..
 * cp[p+1]).  Storage is O(nzc + nnz): the library adds an auxiliary column
 * index of about nzc entries (aux[k] = the first p with jc[p] >= k * 2^s,
 * 2^s about n / nzc) that finds a column in expected constant time, and
 * sizes its per-call x compaction by min(n, nzc).  jc and cp are checked on
 * the host at create time (SPMSPV_ERR_ARG).  x may name any column in [0, n);
 * columns not stored contribute nothing.  The pull direction (which needs the
 * CSC to double as CSR) and spmspv_acl (which reads degrees from column
 * pointers) are not available on a DCSC handle; everything else is.
 */
int spmspv_create_dcsc(spmspv_handle** h, int32_t m, int32_t n, int64_t nnz, int32_t nzc,
                       const int32_t* jc, const int32_t* cp, const int32_t* rowidx, const void* val,
                       int val_type, uint32_t flags);

/*
 * The auxiliary column index spmspv_create_dcsc builds, computed on HOST
 * arrays (no device, no handle): jc host int32[nzc], strictly ascending in
 * [0, n), else SPMSPV_ERR_ARG.  *shift = s, the smallest s >= 0 with
 * n / 2^s <= max(nzc, 1); *aux_len = (n-1)/2^s + 2; aux (host, may be NULL)
 * receives min(aux_capacity, *aux_len) entries, aux[k] = the first position p
 * with jc[p] >= k * 2^s (nzc when there is none).  Column j is stored iff it
 * lies among jc[aux[j >> s] .. aux[(j >> s) + 1]).
 */
int spmspv_dcsc_index(int32_t n, int32_t nzc, const int32_t* jc, int32_t* aux, int64_t aux_capacity,
                      int64_t* aux_len, int32_t* shift);

/* Release the handle and its workspace (synchronises the device). */
int spmspv_destroy(spmspv_handle* h);

/*
 * y <- A (+).(x) x  [under mask]  (Algorithm 1; masks: Sec. V).
 *   semiring    SPMSPV_PLUS_TIMES_F32 | SPMSPV_MIN_SELECT2ND_I32 | SPMSPV_OR_AND_BOOL.
 *   x_idx       device int32[nnz_x], distinct, each in [0, n) (caller contract;
 *               duplicates or out-of-range ids give undefined results).
 *   x_val       device float[] or int32[] per the semiring; may be NULL for
 *               OR_AND_BOOL.
 *   nnz_x       host count, 0 <= nnz_x <= n.  0 gives an empty y.
 *   mask        device uint32[ceil(m/32)] bitmap (bit i%32 of word i/32), or
 *               NULL for no mask.  Without SPMSPV_MASK_COMPLEMENT row i is kept
 *               only where its bit is 1; with it only where its bit is 0.
 *   opts        SPMSPV_MASK_COMPLEMENT | SPMSPV_SORTED_OUT | SPMSPV_SORT_X |
 *               SPMSPV_BUCKETS_ONLY | SPMSPV_X_IDS | SPMSPV_WITH_FEATURES |
 *               schedule bits.  With SPMSPV_SORT_X, repeated or out-of-range x
 *               ids also set SPMSPV_DEV_INDEX.
 *   y_idx       device int32[y_capacity] out.
 *   y_val       device float[]/int32[y_capacity] out (ignored for OR_AND_BOOL).
 *   y_capacity  entries available in y_idx/y_val.  min(m, nnz(A)) always
 *               suffices.  If y needs more, nothing past y_capacity is
 *               written, *d_nnz_y receives the size needed and the device
 *               status gets SPMSPV_DEV_CAPACITY.
 *   d_nnz_y     device int32 out: nnz(y).
 *   stream      CUDA stream.
 * Output order: y_idx is always produced in ascending order (each
 * row-range bucket is emitted in row order and buckets are concatenated in
 * order, Step 3 of Algorithm 1), so SPMSPV_SORTED_OUT costs nothing extra.
 * Direct form: a (+,*) push product with at least 2m products (decided on
 * the device from the work scan) adds every product into a dense accumulator
 * of m floats that the handle keeps in device memory (4m bytes, allocated at
 * create when m <= 2^24; at these sizes it stays in L2), then reads the
 * touched rows back in ascending order and resets them; this replaces the
 * row-range buckets and the shared-memory SPA, with the same index set and
 * values up to the order of the float additions.  SPMSPV_BUCKETS_ONLY keeps
 * the bucketed form for every size.
 */
int spmspv_run(spmspv_handle* h, int semiring, const int32_t* x_idx, const void* x_val,
               int32_t nnz_x, const uint32_t* mask, uint32_t opts, int32_t* y_idx,
               void* y_val, int32_t y_capacity, int32_t* d_nnz_y, spmspv_stream_t stream);

/*
 * The same product with x and y in HOST memory (the end-to-end form): x is
 * copied to device buffers the handle keeps (grown on first use: 8 bytes per
 * x entry and per y entry of capacity), the product runs on `stream` as in
 * spmspv_run, nnz(y) is read back (one synchronisation), then the first
 * min(nnz(y), y_capacity) entries of y are copied out and the stream is
 * synchronised again: on return y and nnz(y) are in host memory.
 *   x_idx, x_val          host arrays as for spmspv_run (page-locked memory
 *                         gives full copy speed; pageable memory works).
 *   mask                  DEVICE bitmap as for spmspv_run, or NULL.
 *   y_idx, y_val          host arrays of y_capacity entries.
 *   nnz_y                 host int32 out: nnz(y) (larger than y_capacity when
 *                         y did not fit, with SPMSPV_DEV_CAPACITY set).
 * Errors as for spmspv_run; calls of this kind on one handle must not
 * overlap (they share the staging buffers).
 */
int spmspv_run_host(spmspv_handle* h, int semiring, const int32_t* x_idx, const void* x_val,
                    int32_t nnz_x, const uint32_t* mask, uint32_t opts, int32_t* y_idx,
                    void* y_val, int32_t y_capacity, int32_t* nnz_y, spmspv_stream_t stream);

/*
 * Breadth-first search from `src` by repeated masked (min, select2nd) SpMSpV
 * (Sec. IV-D; level rule: level[src] = 0, parent[src] = src; every vertex
 * reached at level L has parent = its smallest-id neighbour at level L-1;
 * unreached vertices get -1).  A must be square; for an undirected graph it is
 * symmetric (create with SPMSPV_CSC_PATTERN_SYMMETRIC to allow the pull
 * direction).  Column j's entries are the vertices reached from j.
 *   level, parent  device int32[n] out.
 *   d_nlevels      device int32 out (may be NULL): number of levels (max level + 1).
 *   opts           schedule: SPMSPV_SCHED_OPT(s) for a fixed schedule, SPMSPV_SCHED_AUTO
 *                  for the learned selector (weights must be loaded or trained),
 *                  0 for the default fixed push schedule.
 * The level loop runs on the device (a CUDA graph with a conditional WHILE node,
 * built on first use for each schedule mode): no host synchronisation per level.
 * Allocates the BFS buffers (4 bytes per vertex + a visited bitmap) on first use.
 */
int spmspv_bfs(spmspv_handle* h, int32_t src, int32_t* level, int32_t* parent,
               int32_t* d_nlevels, uint32_t opts, spmspv_stream_t stream);

/*
 * Batched form: B independent products y_b <- A (+).(x) x_b [under mask_b]
 * (no counterpart in the paper; its Sec. I and III-A note that repeated small
 * products are dominated by overhead).  Two forms run it:
 *   persistent  one cooperative kernel launch for the whole batch: its CTAs
 *               scan every frontier, sort each frontier of at most 4096
 *               products in one CTA, run (+,*) frontiers of at least m/2
 *               products in the direct form (products added into dense
 *               accumulators of m floats in device memory, as many at a time
 *               as fit in 128 MB; not with SPMSPV_BUCKETS_ONLY), and the expand
 *               and merge steps of the others with buckets keyed by (frontier,
 *               row block), taking tiles and buckets of all frontiers from
 *               shared device queues.
 *               x_cnt is read on the host first (one synchronisation of
 *               `stream`) to size the work arrays; the launch also needs every
 *               CTA resident (a cooperative launch).  Its buckets hold m/256,
 *               m/128 or m/64 rows by the schedule's width (at most 2^15 rows;
 *               m <= 2^26).
 *   lanes       `lanes` concurrent device-side loops (a graph with conditional
 *               WHILE nodes) that each take the next frontier from a queue and
 *               run the three kernels of spmspv_run on it with their own
 *               workspace (no host synchronisation).
 * Either way y_b has the index set spmspv_run gives for x_b, ascending, and
 * the same values up to the order of the float additions.  All arrays are
 * device arrays:
 *   x_off[B], x_cnt[B]   frontier b is x_idx[x_off[b] .. x_off[b]+x_cnt[b]) and the
 *                        same slice of x_val (ignored for OR_AND_BOOL); each
 *                        0 <= x_cnt[b] <= n, the ids of one frontier distinct.
 *   masks, mask_stride   NULL, or frontier b's complemented mask at
 *                        masks + b*mask_stride (uint32 words, stride >= ceil(m/32));
 *                        opts must then contain SPMSPV_MASK_COMPLEMENT.
 *   y_off[B], y_cap[B]   y_b goes to y_idx/y_val[y_off[b] ..], at most y_cap[b]
 *                        entries (ascending indices); d_nnz_y[b] receives nnz(y_b)
 *                        (the size needed when it exceeds y_cap[b]).
 *   opts                 SPMSPV_SCHED_OPT(s) (pull schedules run as their push
 *                        form), SPMSPV_MASK_COMPLEMENT, SPMSPV_BUCKETS_ONLY.
 *   lanes                0: autotuned: the form and push schedule are taken
 *                        from the handle's tuning cache for this batch profile
 *                        (spmspv_tune_key), or, on the first call with a new
 *                        profile, found by running the batch under every
 *                        candidate (the persistent form under push schedules
 *                        0..5, the lanes form with 4 and 16 lanes under
 *                        schedules 2 and 5; two runs each, the second timed)
 *                        and cached (lanes 0 in the cache: the persistent form).
 *                        Any schedule in opts is then ignored.
 *                        SPMSPV_LANES_PERSISTENT: the persistent form with the
 *                        schedule in opts (or the handle's default).
 *                        1..16: the lanes form with that many lanes; lane
 *                        workspaces (one per lane, as for a handle) and the graph
 *                        are created on first use.
 *                        Forms 0 and SPMSPV_LANES_PERSISTENT synchronise the
 *                        stream, so they must not be captured.
 * Errors: SPMSPV_ERR_ARG for a bad argument (an x_cnt outside [0, n] is found
 * on the host in the persistent form), SPMSPV_ERR_UNSUPPORTED for a batch of
 * 2^31 or more x entries or tiles, SPMSPV_ERR_OOM when work arrays cannot
 * grow.  Device-side problems (y too small, repeated ids) are reported by
 * spmspv_device_status.
 */
#define SPMSPV_LANES_PERSISTENT (-1)
int spmspv_run_batched(spmspv_handle* h, int semiring, int32_t B, const int32_t* x_off,
                       const int32_t* x_cnt, const int32_t* x_idx, const void* x_val,
                       const uint32_t* masks, int64_t mask_stride, uint32_t opts,
                       const int32_t* y_off, const int32_t* y_cap, int32_t* y_idx, void* y_val,
                       int32_t* d_nnz_y, int32_t lanes, spmspv_stream_t stream);

/*
 * Device-clock durations (ms) of the phases of the handle's last persistent
 * batched launch (spmspv_run_batched, lanes 0 or SPMSPV_LANES_PERSISTENT):
 * ms[0] work scan, ms[1] plan, ms[2] tile starts, ms[3] expand (Step 1 and
 * the one-CTA small frontiers, summed over the bucket waves), ms[4] merge
 * (Steps 2-3, summed over the bucket waves), ms[5] the whole launch, ms[6]
 * the direct form's expand and ms[7] its compaction (summed over its waves);
 * min(capacity, 8) entries are written.  *waves (may be NULL) receives the
 * launch's number of bucket waves.
 * Synchronises the handle's last stream.  SPMSPV_ERR_STATE before any such
 * launch.
 */
int spmspv_batched_phase_times(spmspv_handle* h, double* ms, int32_t capacity, int32_t* waves);

/*
 * Multi-source BFS: B searches (the BFS of spmspv_bfs from each of sources[B],
 * device array) advanced together, one batched step per level.
 *   level, parent  device int32[B][n] out (row b = search from sources[b]).
 *   nlevels        device int32 out (may be NULL): levels of the deepest search.
 *   opts, lanes    as for spmspv_run_batched: a push schedule; 1..16 lanes;
 *                  SPMSPV_LANES_PERSISTENT, every level one persistent launch
 *                  over all sources (y_b = A x_b with x_b the frontier carrying
 *                  its vertex ids, under the complement of visited_b); or 0 for
 *                  autotuned: the first call with a new B profile runs the whole
 *                  search under every candidate (lanes 2/4/8/16 and the
 *                  persistent form, each with every push schedule), timed, and
 *                  caches the fastest.
 *                  SPMSPV_SCHED_AUTO (weights set, pattern-symmetric handle):
 *                  the learned schedule picks push or pull per source and level,
 *                  as in spmspv_bfs (in the persistent form the sources that
 *                  pull run in one batched pull kernel beside the push launch;
 *                  lanes 0: only the form and lane count are tuned); levels and
 *                  parents are the same either way.  It adds B*n/4 bytes of
 *                  frontier bitmaps (the persistent form B*n/8).
 * Allocates B*(4n + n/8) bytes of frontiers and visited bitmaps for the call
 * (the persistent form 8*B*n more: the level's product and its parents);
 * synchronises the stream once per level to test for termination (the
 * persistent form twice: its launch reads the frontier sizes first).
 */
int spmspv_msbfs(spmspv_handle* h, int32_t B, const int32_t* sources, int32_t* level,
                 int32_t* parent, int32_t* nlevels, uint32_t opts, int32_t lanes,
                 spmspv_stream_t stream);

/*
 * Connected components of an undirected graph (square, pattern-symmetric
 * handle) by minimum-label propagation, one (select2nd, min) SpMSpV per round
 * on the vertices whose label dropped in the previous round (Sec. I lists
 * connected components as an SpMSpV customer; the algorithm is this
 * library's reading).  On return labels[v] is the smallest vertex id of v's
 * component.  All rounds run in one CUDA graph launch; asynchronous on
 * `stream`.
 *   labels     device int32[n] out.
 *   d_nrounds  device int32 out (may be NULL): rounds run (the last finds nothing).
 *   opts       SPMSPV_SCHED_OPT(s) with a push schedule s in 0..5, or 0 for the
 *              default; SPMSPV_SCHED_AUTO is UNSUPPORTED.
 * Allocates 16 bytes per vertex of frontier buffers on first use.
 */
int spmspv_cc(spmspv_handle* h, int32_t* labels, int32_t* d_nrounds, uint32_t opts,
              spmspv_stream_t stream);

/*
 * Maximal independent set of an undirected graph (square, pattern-symmetric
 * handle) by Luby's rounds with fixed priorities (Sec. I lists maximal
 * independent sets as an SpMSpV customer; the rounds are this library's
 * reading).  Per round, with C the undecided vertices: y = A (min.select2nd)
 * prio|C with rows masked to C; the v in C with v not in y or prio(v) <= y(v)
 * join; z = A (or.and) joiners with rows masked to the still undecided; z
 * leaves C.  Until C is empty.  With distinct priorities the set is the
 * greedy one in priority order (smallest first).  Self loops are ignored.
 * All rounds run in one CUDA graph launch; asynchronous on `stream`.
 *   prio       device int32[n] in: priorities, which must be distinct (for
 *              example a permutation); repeated values end the rounds all the
 *              same but may put two adjacent vertices in the set.
 *   in_set     device int32[n] out: 1 for members, 0 otherwise.
 *   d_nrounds  device int32 out (may be NULL): rounds run.
 *   opts       SPMSPV_SCHED_OPT(s) with a push schedule s in 0..5, or 0 for the
 *              default; SPMSPV_SCHED_AUTO is UNSUPPORTED.
 * Allocates about 24 bytes per vertex of work buffers on first use.
 */
int spmspv_mis(spmspv_handle* h, const int32_t* prio, int32_t* in_set, int32_t* d_nrounds,
               uint32_t opts, spmspv_stream_t stream);

/*
 * Maximum-cardinality matching of the bipartite graph between the m rows and
 * the n columns of A (an edge wherever A(i,j) is stored; any shape, no
 * symmetry needed) by phases of multi-source alternating BFS, one
 * (min.select2nd) SpMSpV per level with the visited rows as a complemented
 * mask (Sec. I lists bipartite matching as an SpMSpV customer; the phases are
 * this library's reading).  A phase grows one BFS tree from every free column,
 * keeps the first free row each tree reaches and flips those vertex-disjoint
 * augmenting paths; the search ends when a phase finds none, and the matching
 * is then maximum.  Which maximum matching comes out depends on the order of
 * atomic operations; its cardinality does not.  All phases run in one CUDA
 * graph launch; asynchronous on `stream`.
 *   mate_r     device int32[m] out: matched column of each row, or -1.
 *   mate_c     device int32[n] out: matched row of each column, or -1.
 *   d_card     device int32 out (may be NULL): the cardinality.
 *   d_nphases  device int32 out (may be NULL): phases that flipped paths.
 *   opts       SPMSPV_SCHED_OPT(s) with a push schedule s in 0..5, or 0 for the
 *              default; SPMSPV_SCHED_AUTO is UNSUPPORTED.
 * SPMSPV_DEV_BOUND in the device status afterwards means a loop bound was
 * reached and the outputs are invalid.  Allocates about 16 bytes per row and
 * 16 per column of work buffers on first use.
 */
int spmspv_mcm(spmspv_handle* h, int32_t* mate_r, int32_t* mate_c, int32_t* d_card,
               int32_t* d_nphases, uint32_t opts, spmspv_stream_t stream);

/*
 * Andersen-Chung-Lang push from B seeds (device int32[B]) on the unweighted
 * graph (handle created with SPMSPV_VAL_NONE; A symmetric), one batched (+,*)
 * SpMSpV per step (Sec. I lists ACL as a one-SpMSpV-per-step customer; the
 * paper gives no algorithm, so the synchronous form below is this library's
 * reading).  Per seed b: r = e_seed, p = 0; each step, with d(u) = column
 * length and S = {u : r(u) >= eps*d(u)}: x(u) = (1-alpha) r(u) / (2 d(u)) and
 * p(u) += alpha r(u), r(u) = (1-alpha) r(u) / 2 for u in S, then r += A x.
 * Stops when every S is empty or after max_steps steps.  sum(p) + sum(r) stays 1.
 * 1 <= B <= 65535 and B*n < 2^31, else SPMSPV_ERR_UNSUPPORTED.
 *   p_out, r_out  device float[B][n] out.   steps_out  device int32 out (may be NULL).
 *   lanes   1..16 concurrent lanes with the handle's default schedule,
 *           SPMSPV_LANES_PERSISTENT (each step's products one persistent launch
 *           over every seed), or 0 for autotuned (as for spmspv_msbfs: whole
 *           runs timed per candidate, lanes and persistent form).
 * Allocates about 20 B*n bytes of work arrays for the call; synchronises the
 * stream once per step (the persistent form twice).
 */
int spmspv_acl(spmspv_handle* h, int32_t B, const int32_t* seeds, float alpha, float eps,
               int32_t max_steps, float* p_out, float* r_out, int32_t* steps_out, int32_t lanes,
               spmspv_stream_t stream);

/* ---- autotuner of the batched form (no counterpart in the paper) ----
 * The cache lives in the handle (lost at spmspv_destroy).  A profile key packs
 * kind (0 batched SpMSpV, 1 multi-source BFS, 2 ACL, 3 multi-source BFS with
 * the learned schedule: lanes only, schedule entry 0), semiring, whether masks
 * are given, ceil(log2 B) and ceil(log2(1 + total nnz(x) / B)); calls whose
 * profiles share a key share one tuning.  spmspv_tune_key is pure host code.
 */
uint64_t spmspv_tune_key(int kind, int semiring, int masked, int32_t B, int64_t total_nnz_x);
/* What the handle's last lanes = 0 call ran with (lanes 0: the persistent
 * form); from_cache = 1 when no timing was needed.  SPMSPV_ERR_STATE before
 * any such call. */
int spmspv_last_tuned(spmspv_handle* h, int32_t* lanes, int32_t* sched, int32_t* from_cache);
/* Copy up to `capacity` cache entries out (host arrays, any may be NULL);
 * *count receives the number of entries.  ms is the timed run (NaN if set). */
int spmspv_tune_entries(spmspv_handle* h, uint64_t* keys, int32_t* lanes, int32_t* sched,
                        float* ms, int32_t capacity, int32_t* count);
/* Seed or override an entry (lanes 1..16, or 0 for the persistent form;
 * push schedule 0..5). */
int spmspv_tune_set(spmspv_handle* h, uint64_t key, int32_t lanes, int32_t sched);
int spmspv_tune_clear(spmspv_handle* h);

/* ---- learned schedule selector ----
 * No counterpart in the paper, which leaves open when to switch between the
 * vector-driven (push) and matrix-driven (pull) forms (Sec. V).  A 6->32->32->12
 * FP32 MLP predicts the log run time of each of the 12 schedules
 * (SPMSPV_SCHED_ID = dir*6 + quantum*3 + width: 3 bucket widths x 2 work quanta x
 * {push, pull}) from features of the call (log2(1+nnz(x)), log2(1+work), max/mean
 * selected column length, fraction of rows set in the mask, log2(m), nnz(A)/n) computed on the
 * device after the work scan, and picks the fastest predicted allowed schedule
 * (pull only for symmetric patterns).  It never changes results.
 * Parameters: SPMSPV_SELECTOR_NPARAM floats = W1[32][6] b1[32] W2[32][32] b2[32]
 * W3[12][32] b3[12] mean[6] scale[6] (inputs are (feature - mean) * scale). */
#define SPMSPV_SELECTOR_NPARAM 1688

/* Install / read the selector parameters (host arrays of `n` floats). */
int spmspv_selector_set(spmspv_handle* h, const float* params, int32_t n);
/* Install the selector parameters from a weights file: a JSON object whose
 * "params" member is an array of SPMSPV_SELECTOR_NPARAM numbers (the format
 * paper_1610_07902_gb300/selector_weights.json has; other members are
 * ignored).  `path` is a host string owned by the caller.  A missing file, a
 * missing or malformed array or a wrong count returns SPMSPV_ERR_ARG and
 * leaves the installed parameters as they were.  Synchronous. */
int spmspv_selector_load(spmspv_handle* h, const char* path);
int spmspv_selector_get(spmspv_handle* h, float* params, int32_t n);

/* The 6 selector features of the handle's last call (host out; synchronises). */
int spmspv_last_features(spmspv_handle* h, float* feats);

/* The plain fixed schedule: what spmspv_run uses without SPMSPV_SCHED_FORCE or
 * SPMSPV_SCHED_AUTO, and the AUTO fallback before weights are set. */
int spmspv_default_schedule(spmspv_handle* h, int32_t* sched);
/* Schedule id the selector chose in the handle's last SPMSPV_SCHED_AUTO call, or
 * the id of the last forced schedule (host out; synchronises). */
int spmspv_last_schedule(spmspv_handle* h, int32_t* sched);

/* Train the selector on the device with the library's own forward/backward
 * kernels and Adam: feats [n][6] raw features, target [n][12] log run times,
 * valid [n][12] bytes (NULL: all valid), all device pointers.  Starts from the
 * installed parameters, else a seeded He initialisation; the input
 * normalisation is taken from the data.  loss (host, `epochs` floats, may be
 * NULL) receives the mean squared error of each epoch.  Synchronous. */
int spmspv_selector_train(spmspv_handle* h, const float* feats, const float* target,
                          const uint8_t* valid, int32_t n, int32_t epochs, int32_t batch,
                          float lr, uint64_t seed, float* loss);

/* Gradient (host out, 1676 floats: the weights in parameter order) and loss
 * (host out, may be NULL) of the summed squared error at the installed
 * parameters, on device arrays as for spmspv_selector_train.  Synchronous. */
int spmspv_selector_grad(spmspv_handle* h, const float* feats, const float* target,
                         const uint8_t* valid, int32_t n, float* grad, float* loss);

/* Failure-detection self-test (no counterpart in the paper): runs one warp
 * of the scan's decoupled look-back against a predecessor that never
 * publishes, with its wait bounded by `spins` iterations (1 .. 2^22), so that
 * the wait gives up; synchronous on `stream`.  Afterwards
 * spmspv_device_status() reports SPMSPV_DEV_TIMEOUT and the handle keeps
 * working: no fault, no trap, no hang. */
int spmspv_selftest_wait_timeout(spmspv_handle* h, uint32_t spins, spmspv_stream_t stream);

/* Device status word of the handle: synchronises the handle's last stream,
 * returns the SPMSPV_DEV_* bits in *flags (host out) and clears them.  The
 * bits of the batched form's lanes (their own workspaces) are included. */
int spmspv_device_status(spmspv_handle* h, uint32_t* flags);

/* Multiply count of the last run (host out, synchronises): the sum of the
 * selected column lengths, the df term of Sec. II-D, before masking. */
int spmspv_last_work(spmspv_handle* h, int64_t* work);

/*
 * y <- A (+).(x) x without a handle and without allocating device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc, such as code that must not stall the device
 * (cudaMalloc can synchronise it), code running inside a host process whose
 * allocator owns all device memory, or code with a device-memory budget fixed
 * at load time.  The caller passes the CSC matrix, x and y (device pointers,
 * caller-owned, same meaning and layout as spmspv_create_csc + spmspv_run);
 * the scratch the product needs (buckets, compacted x, scan state) lives in
 * one file-scope device array of about 7 MB that the library holds on every
 * GPU that loads it, until the process exits.
 *   Limits (rejected with SPMSPV_ERR_UNSUPPORTED and a message naming the
 *   limit): m <= 2^22 rows, nnz(A) <= 2^20, nnz_x <= 2^16.  Only the default
 *   schedule: SPMSPV_SCHED_* options are rejected the same way.
 *   val_type: SPMSPV_VAL_F32 or SPMSPV_VAL_NONE, as for spmspv_create_csc.
 *   Output order, capacity rule and *d_nnz_y: as for spmspv_run (a y that does
 *   not fit leaves the size it needs in *d_nnz_y).
 *   No handle checks the matrix here, so every call makes one pass over A's
 *   nnz row ids to size the bucket regions (a call costs O(nnz(A)) on top of
 *   the product's own work).  A row id outside [0, m), or an x index that is
 *   out of range or repeated, is dropped without any access outside the
 *   arrays and the call reports it by setting *d_nnz_y to -1 (y undefined).
 * The first call on a device looks up the array's device address with that
 * device current (a one-time set-up); make that first call before any stream
 * capture.  The address is cached per device for the life of the process: a
 * process that calls cudaDeviceReset must not call this entry point on that
 * device afterwards.  Every call shares the one array and each call clears the part that
 * must start at zero: calls whose kernels overlap on the GPU (other streams,
 * or other host threads without ordering) race on it and give undefined
 * results.  Asynchronous on `stream`; nothing is allocated or freed.
 */
int spmspv_run_noalloc(int32_t m, int32_t n, int64_t nnz, const int32_t* colptr,
                       const int32_t* rowidx, const void* val, int val_type, int semiring,
                       const int32_t* x_idx, const void* x_val, int32_t nnz_x,
                       const uint32_t* mask, uint32_t opts, int32_t* y_idx, void* y_val,
                       int32_t y_capacity, int32_t* d_nnz_y, spmspv_stream_t stream);

/* ---- per-stage timing (CUDA events on the launch stream) ----
 * Stage ids of spmspv_profile_end's stage_ms array. */
#define SPMSPV_STAGE_SCAN 0    /* K1 work scan (Algorithm 2's role) */
#define SPMSPV_STAGE_SELECT 1  /* learned schedule selector */
#define SPMSPV_STAGE_SCATTER 2 /* K2 expand + multiply + bucket (Step 1) */
#define SPMSPV_STAGE_MERGE 3   /* K3 SPA merge + concatenation (Steps 2-3) */
#define SPMSPV_STAGE_PULL 4    /* pull direction (matrix-driven) kernels */
#define SPMSPV_NUM_STAGES 5

/* Start recording a CUDA event before and after every stage of every
 * following call on this handle (adds a few microseconds per call). */
int spmspv_profile_begin(spmspv_handle* h);

/* Stop recording; synchronise; stage_ms (host out, n_stages entries) gets
 * the summed device time of each stage over the recorded calls and
 * *n_calls (host out, may be NULL) the number of calls. */
int spmspv_profile_end(spmspv_handle* h, double* stage_ms, int32_t n_stages, int32_t* n_calls);

#ifdef __cplusplus
}
#endif
#endif /* SPMSPV_H_ */
