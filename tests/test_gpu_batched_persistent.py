"""The persistent one-launch batched form (spmspv_run_batched with lanes
SPMSPV_LANES_PERSISTENT or 0) against the oracle: every frontier's y must
equal the single product's (index sets and integer values bit for bit, FP32
values within the parity tolerance).  Covers the three frontier kinds (no
products, at most 4096 products sorted by one CTA, larger ones through the
(frontier, row block) buckets), both work quanta and several bucket widths,
masks, more waves than one, repeated launches, y capacities, DCSC."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import SEMIRING_TO_ORACLE, compare, mask_bits, need_gpu, x_values

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = need_gpu()
    from paper_1610_07902_gb300 import spmspv as S
    S.load()
    return torch, S


def pack(fronts):
    x_cnt = np.array([f[0].shape[0] for f in fronts], np.int32)
    x_off = np.concatenate([[0], np.cumsum(x_cnt)[:-1]]).astype(np.int32)
    x_idx = np.concatenate([f[0] for f in fronts] + [np.zeros(1, np.int32)]).astype(np.int32)
    return x_cnt, x_off, x_idx


def run_and_check(torch, S, A, Ad, fronts, semiring, lanes, opts=0, masks_u8=None, y_cap=None, label=""):
    B = len(fronts)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    x_cnt, x_off, x_idx = pack(fronts)
    xs = [x_values(semiring, xi, xf) for xi, xf in fronts]
    xv = None if semiring == 2 else dev(np.concatenate(xs + [np.zeros(1, xs[0].dtype)]))
    cap = np.full(B, A.m, np.int32) if y_cap is None else y_cap
    y_off = (np.arange(B, dtype=np.int64) * A.m).astype(np.int32)
    yi = torch.full((B * A.m,), -7, dtype=torch.int32, device="cuda")
    vdt = torch.float32 if semiring == 0 else torch.int32
    yv = None if semiring == 2 else torch.zeros(B * A.m, dtype=vdt, device="cuda")
    nz = torch.full((B,), -1, dtype=torch.int32, device="cuda")
    words = (A.m + 31) // 32
    msk = None
    if masks_u8 is not None:
        msk = dev(np.concatenate([mask_bits(mm) for mm in masks_u8]).view(np.int32))
        opts |= S.SPMSPV_MASK_COMPLEMENT
    S.spmspv_run_batched(Ad.handle, semiring, B, dev(x_off), dev(x_cnt), dev(x_idx), xv, msk, words, opts,
                         dev(y_off), dev(cap), yi, yv, nz, lanes)
    nz_h, yi_h = nz.cpu().numpy(), yi.cpu().numpy()
    yv_h = None if yv is None else yv.cpu().numpy()
    over = False
    for b in range(B):
        ref = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, SEMIRING_TO_ORACLE[semiring], fronts[b][0], xs[b],
                            None if masks_u8 is None else masks_u8[b], True)
        k = ref.idx.shape[0]
        assert nz_h[b] == k, (label, semiring, b, nz_h[b], k)
        o = int(y_off[b])
        if k > cap[b]:
            over = True
            np.testing.assert_array_equal(yi_h[o:o + cap[b]], ref.idx[:cap[b]])
            assert (yi_h[o + cap[b]:o + cap[b] + 8] == -7).all()  # nothing past the capacity
            continue
        compare(semiring, ref, yi_h[o:o + k], None if yv_h is None else yv_h[o:o + k])
        assert (yi_h[o + k:o + k + 4] == -7).all()
    st = S.spmspv_device_status(Ad.handle)
    assert st == (S.SPMSPV_DEV_CAPACITY if over else 0), (label, st)


def mixed_fronts(n, B, seed, fmax):
    rng = np.random.default_rng(seed)
    sizes = np.maximum(1, np.floor(10 ** rng.uniform(0, np.log10(fmax), B))).astype(np.int64)
    sizes[::7] = 0  # empty frontiers among the others
    out = []
    for b, s in enumerate(sizes):
        if s == 0:
            out.append((np.zeros(0, np.int32), np.zeros(0, np.float32)))
        else:
            out.append(synth.frontier(n, int(min(s, n)), seed=seed * 1000 + b))
    return out


@pytest.mark.parametrize("sched", [0, 2, 4, 5])
@pytest.mark.parametrize("masked", [False, True])
@pytest.mark.parametrize("buckets_only", [False, True])
def test_persistent_matches_oracle(lib, sched, masked, buckets_only):
    """(+,*) frontiers of at least m/2 products run in the direct form unless
    SPMSPV_BUCKETS_ONLY is given; both are compared."""
    torch, S = lib
    A = synth.rmat(14, seed=4)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val)
    fronts = mixed_fronts(A.n, 40, 11 + sched, 5000)
    W = [int(np.diff(A.colptr)[f[0]].sum()) for f in fronts]
    assert sum(w >= A.m // 2 for w in W) >= 5
    rng = np.random.default_rng(sched)
    masks = [(rng.random(A.m) < 0.3).astype(np.uint8) for _ in fronts] if masked else None
    extra = S.SPMSPV_BUCKETS_ONLY if buckets_only else 0
    for semiring in (0, 1, 2):
        run_and_check(torch, S, A, Ad, fronts, semiring, S.SPMSPV_LANES_PERSISTENT,
                      S.SPMSPV_SCHED_OPT(sched) | extra, masks, label="sched %d" % sched)
    Ad.close()


def test_persistent_waves_and_repeats(lib):
    """Large frontiers whose products add up to many times nnz(A): the first
    launch splits them into waves (its window is one matrix), the second runs
    them in one wave; both must be exact."""
    torch, S = lib
    A = synth.rmat(12, seed=21)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val)
    fronts = []
    for b in range(30):
        k = [3000, 3, 0, 2000, 40][b % 5]
        fronts.append(synth.frontier(A.n, k, seed=500 + b) if k else (np.zeros(0, np.int32), np.zeros(0, np.float32)))
    W = sum(int(np.diff(A.colptr)[f[0]].sum()) for f in fronts)
    assert W > 3 * A.nnz  # several waves at the first launch
    waves = []
    for call in range(3):
        run_and_check(torch, S, A, Ad, fronts, 0, S.SPMSPV_LANES_PERSISTENT,
                      S.SPMSPV_SCHED_OPT(5) | S.SPMSPV_BUCKETS_ONLY, label="call %d" % call)
        ms, w = S.spmspv_batched_phase_times(Ad.handle)
        parts = ms[[0, 1, 2, 3, 4, 6, 7]].sum()
        assert (ms >= 0).all() and abs(parts - ms[5]) <= 1e-3 * ms[5] + 1e-3
        waves.append(w)
    assert waves[0] > 1 and waves[1] == 1 and waves[2] == 1, waves
    run_and_check(torch, S, A, Ad, fronts, 1, S.SPMSPV_LANES_PERSISTENT, S.SPMSPV_SCHED_OPT(1))
    Ad.close()


def regular_matrix(n, d, seed):
    """n x n, every column d distinct random rows (ascending), random values."""
    rng = np.random.default_rng(seed)
    # d distinct blocks of 8 rows per column, one row from each
    rows = np.argsort(rng.random((n, n // 8)), axis=1)[:, :d] * 8 + rng.integers(0, 8, (n, d))
    rowidx = np.sort(rows, axis=1).astype(np.int32).ravel()
    colptr = (np.arange(n + 1) * d).astype(np.int32)
    val = rng.uniform(-1, 1, rowidx.shape[0]).astype(np.float32)
    return synth.CSC(n, n, colptr, rowidx, val, "regular")


def test_persistent_boundaries(lib):
    """Frontiers of exactly 4096 products (the largest sorted by one CTA),
    4097 (the smallest through buckets), one product, a tile boundary inside
    a column, and y capacities below nnz(y) for both kinds."""
    torch, S = lib
    A = regular_matrix(8192, 16, 3)
    deg = np.diff(A.colptr)
    assert (deg == 16).all()
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val)
    rng = np.random.default_rng(5)
    perm = rng.permutation(A.n).astype(np.int32)

    def fr(lo, k):
        idx = np.sort(perm[lo:lo + k])
        return idx, rng.uniform(-1, 1, k).astype(np.float32)
    fronts = [fr(0, 256), fr(300, 257), fr(600, 1), fr(700, 512), fr(1300, 513), fr(2000, 255), fr(2400, 700)]
    for semiring in (0, 1, 2):
        for sched in (0, 5):
            run_and_check(torch, S, A, Ad, fronts, semiring, S.SPMSPV_LANES_PERSISTENT, S.SPMSPV_SCHED_OPT(sched))
    cap = np.full(len(fronts), A.m, np.int32)
    cap[0] = 100   # a sorted frontier
    cap[4] = 1000  # a bucketed one
    run_and_check(torch, S, A, Ad, fronts, 0, S.SPMSPV_LANES_PERSISTENT, S.SPMSPV_SCHED_OPT(5), y_cap=cap)
    # a batch without any x entry, and one of a single frontier
    empty = [(np.zeros(0, np.int32), np.zeros(0, np.float32))] * 3
    run_and_check(torch, S, A, Ad, empty, 0, S.SPMSPV_LANES_PERSISTENT)
    run_and_check(torch, S, A, Ad, fronts[4:5], 0, S.SPMSPV_LANES_PERSISTENT)
    Ad.close()


def test_persistent_empty_columns_and_dcsc(lib):
    """x entries whose columns hold nothing (dropped by the scan), on a CSC
    and on the DCSC form of the same hypersparse matrix."""
    torch, S = lib
    n = 1 << 16
    full = synth.rmat(12, seed=6)
    rng = np.random.default_rng(8)
    cols = np.sort(rng.choice(n, full.n, replace=False)).astype(np.int32)
    colptr = np.zeros(n + 1, np.int64)
    colptr[cols + 1] = np.diff(full.colptr)
    colptr = np.cumsum(colptr).astype(np.int32)
    A = synth.CSC(n, n, colptr, full.rowidx * 16, full.val, "hyper")
    fronts = []
    for b in range(12):
        k = [5, 300, 2000, 40][b % 4]
        idx = np.sort(rng.choice(n, k, replace=False)).astype(np.int32)
        fronts.append((idx, rng.uniform(-1, 1, k).astype(np.float32)))
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val)
    for semiring in (0, 1):
        run_and_check(torch, S, A, Ad, fronts, semiring, S.SPMSPV_LANES_PERSISTENT)
    Ad.close()
    nzc = cols.shape[0]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    jc, cp = dev(cols), dev(full.colptr.astype(np.int32))
    ri, va = dev(A.rowidx), dev(A.val)
    h = S.spmspv_create_dcsc(A.m, A.n, A.nnz, nzc, jc, cp, ri, va)

    class D:
        handle = h
    for semiring in (0, 2):
        run_and_check(torch, S, A, D, fronts, semiring, S.SPMSPV_LANES_PERSISTENT)
    S.spmspv_destroy(h)


def test_persistent_autotuned_caches_schedule(lib):
    torch, S = lib
    A = synth.rmat(13, seed=9)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val)
    fronts = mixed_fronts(A.n, 24, 31, 3000)
    for call in range(2):
        run_and_check(torch, S, A, Ad, fronts, 0, 0)
        lanes, sched, cached = S.spmspv_last_tuned(Ad.handle)
        assert lanes in (0, 4, 16) and 0 <= sched < 6 and cached == (call == 1)
    Ad.close()


def test_persistent_direct_form_waves_and_reuse(lib):
    """Many frontiers in the direct form (more than one wave of accumulators
    on a matrix of 2^20 rows, 32 per wave), mixed with bucketed and sorted
    ones, twice in a row (the accumulators must be clean after a launch), and
    with y capacities below nnz(y) in the direct form."""
    torch, S = lib
    A = synth.rmat(20, seed=9)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val)
    deg = np.diff(A.colptr)
    rng = np.random.default_rng(2)
    fronts = []
    for b in range(70):
        k = [40000, 60000, 50000, 45000, 30, 2000, 1][b % 7]
        fronts.append(synth.frontier(A.n, k, seed=700 + b))
    W = [int(deg[f[0]].sum()) for f in fronts]
    assert sum(w >= A.m // 2 for w in W) > 32
    for call in range(2):
        run_and_check(torch, S, A, Ad, fronts, 0, S.SPMSPV_LANES_PERSISTENT, S.SPMSPV_SCHED_OPT(5),
                      label="call %d" % call)
    cap = np.full(len(fronts), A.m, np.int32)
    cap[0] = 5000
    cap[3] = 17
    run_and_check(torch, S, A, Ad, fronts, 0, S.SPMSPV_LANES_PERSISTENT, S.SPMSPV_SCHED_OPT(5), y_cap=cap)
    run_and_check(torch, S, A, Ad, fronts[:6], 0, S.SPMSPV_LANES_PERSISTENT, S.SPMSPV_SCHED_OPT(2))
    Ad.close()


def test_persistent_msbfs_and_plus_share_accumulators(lib):
    """The direct form's accumulators hold -0.0 in every row for (+,*) and
    INT32_MAX for the multi-source BFS ((min, select2nd) with vertex ids):
    alternating the two on one handle must leave both exact (every search
    against the reference, more sources than one wave of accumulators)."""
    torch, S = lib
    A = synth.rmat(16, seed=13)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
    deg = np.diff(A.colptr)
    fronts = [synth.frontier(A.n, [9000, 12000, 40, 1][b % 4], seed=900 + b) for b in range(24)]
    assert sum(int(deg[f[0]].sum()) >= A.m // 2 for f in fronts) >= 10
    srcs = synth.sources(A.colptr, 40, seed=17).astype(np.int32)
    B = srcs.shape[0]
    refs = [oracle.bfs(A.colptr, A.rowidx, int(s))[:2] for s in srcs]
    for rep in range(2):
        run_and_check(torch, S, A, Ad, fronts, 0, S.SPMSPV_LANES_PERSISTENT, S.SPMSPV_SCHED_OPT(5),
                      label="plus %d" % rep)
        level = torch.empty(B * A.n, dtype=torch.int32, device="cuda")
        parent = torch.empty(B * A.n, dtype=torch.int32, device="cuda")
        S.spmspv_msbfs(Ad.handle, B, torch.from_numpy(srcs).cuda(), level, parent, None,
                       S.SPMSPV_SCHED_OPT(2 + 3 * rep), S.SPMSPV_LANES_PERSISTENT)
        lv = level.cpu().numpy().reshape(B, A.n)
        pa = parent.cpu().numpy().reshape(B, A.n)
        for b in range(B):
            np.testing.assert_array_equal(lv[b], refs[b][0], err_msg="levels of source %d" % b)
            np.testing.assert_array_equal(pa[b], refs[b][1], err_msg="parents of source %d" % b)
        assert S.spmspv_device_status(Ad.handle) == 0
    Ad.close()
