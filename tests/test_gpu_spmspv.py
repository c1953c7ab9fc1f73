"""GPU parity: the CUDA SpMSpV path through the C ABI against the CPU oracle.

Index sets and (min, select2nd) values must match bit for bit; (+,*) values
must satisfy |y_gpu - y_fp64| <= 1e-5 * sum_j |A(i,j) x(j)| (gpu_util.FP_TOL).
Inputs are seeded synthetic graphs of the shapes the paper evaluates on:
Erdos-Renyi (the Sec. II-A model), scale-free R-MAT and high-diameter grids
(the two classes of Table IV).
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import FP_TOL, SEMIRING_TO_ORACLE, compare, mask_bits, need_gpu, x_values

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = need_gpu()
    from paper_1610_07902_gb300 import spmspv as S
    S.load()
    return torch, S


def _run(lib, A, Ad, semiring, x_idx, x_val, mask_u8=None, complement=True, sched=None,
         cap=None, auto=False, extra_opts=0):
    torch, S = lib
    dev = "cuda"
    xi = torch.from_numpy(np.ascontiguousarray(x_idx, np.int32)).to(dev)
    xv = None
    if x_val is not None:
        xv = torch.from_numpy(np.ascontiguousarray(x_val)).to(dev)
    mask = None
    opts = S.SPMSPV_SORTED_OUT | extra_opts
    if mask_u8 is not None:
        mask = torch.from_numpy(mask_bits(mask_u8).view(np.int32)).to(dev)
        if complement:
            opts |= S.SPMSPV_MASK_COMPLEMENT
    if sched is not None:
        opts |= S.SPMSPV_SCHED_OPT(sched)
    if auto:
        opts |= S.SPMSPV_SCHED_AUTO
    yi, yv, k = Ad.multiply(semiring, xi, xv, mask, opts, y_capacity=cap)
    st = S.spmspv_device_status(Ad.handle)
    return (yi.cpu().numpy(), None if yv is None else yv.cpu().numpy(), k, st)


def _check(lib, A, Ad, semiring, x_idx, xf, mask_u8=None, complement=True, sched=None, extra_opts=0):
    xv = x_values(semiring, x_idx, xf)
    ref = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, SEMIRING_TO_ORACLE[semiring], x_idx,
                        xv, mask_u8, complement)
    yi, yv, k, st = _run(lib, A, Ad, semiring, x_idx, xv, mask_u8, complement, sched,
                         extra_opts=extra_opts)
    assert st == 0, "device status %d" % st
    assert k == ref.idx.shape[0]
    worst = compare(semiring, ref, yi, yv)
    _, S = lib
    assert S.spmspv_last_work(Ad.handle) == ref.nmult
    if semiring == 0 and not (extra_opts & S.SPMSPV_BUCKETS_ONLY):
        # (+,*) calls with many products run the direct form: the bucketed one too
        worst = max(worst, _check(lib, A, Ad, semiring, x_idx, xf, mask_u8, complement, sched,
                                  extra_opts | S.SPMSPV_BUCKETS_ONLY))
    return worst


def _dev_matrix(lib, A, flags=0):
    _, S = lib
    return S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val, flags=flags)


def test_hand_worked_example(lib):
    from golden_util import load_hand_example
    import synth as _s
    g = load_hand_example()
    A = _s.CSC(g["m"], g["n"], g["colptr"], g["rowidx"], g["val"])
    Ad = _dev_matrix(lib, A)
    xi = np.array(g["x_idx"], np.int32)
    yi, yv, k, st = _run(lib, A, Ad, 0, xi, np.array(g["x_val_plus_times"], np.float32))
    assert list(yi) == g["expect_plus_times"]["idx"] and list(yv) == g["expect_plus_times"]["val"]
    yi, yv, k, st = _run(lib, A, Ad, 1, xi, np.array(g["x_val_min_select2nd"], np.int32))
    assert list(yi) == g["expect_min_select2nd"]["idx"] and list(yv) == g["expect_min_select2nd"]["val"]
    yi, yv, k, st = _run(lib, A, Ad, 2, xi, None)
    assert list(yi) == g["expect_or_and"]["idx"]
    mask = np.zeros(g["m"], np.uint8)
    mask[g["mask_rows"]] = 1
    yi, yv, k, st = _run(lib, A, Ad, 0, xi, np.array(g["x_val_plus_times"], np.float32), mask, True)
    assert list(yi) == g["expect_plus_times_complement_mask"]["idx"]
    assert list(yv) == g["expect_plus_times_complement_mask"]["val"]
    yi, yv, k, st = _run(lib, A, Ad, 0, xi, np.array(g["x_val_plus_times"], np.float32), mask, False)
    assert list(yi) == g["expect_plus_times_structural_mask"]["idx"]
    Ad.close()


def test_erdos_renyi_config(lib):
    """n = 65,536, 16 nnz per column on average, 655 random x entries (1%)."""
    A = synth.erdos_renyi(65536, d=16, seed=1)
    Ad = _dev_matrix(lib, A)
    x_idx, xf = synth.frontier(A.n, 655, seed=1, stream=2)
    for semiring in (0, 1, 2):
        _check(lib, A, Ad, semiring, x_idx, xf)
    Ad.close()


@pytest.mark.parametrize("shape", [(1, 1), (1, 50), (50, 1), (100, 300), (300, 100),
                                   (1000, 1000), (5000, 77), (70000, 900)])
@pytest.mark.parametrize("semiring", [0, 1, 2])
def test_random_shapes_all_schedules(lib, shape, semiring):
    m, n = shape
    rng = np.random.default_rng(m * 7919 + n)
    d = min(12.0, max(1.0, m * 0.3))
    A = synth.erdos_renyi(n, d=d, m=m, seed=m + n) if m > 1 else synth.CSC(
        1, n, np.arange(n + 1, dtype=np.int32), np.zeros(n, np.int32), rng.random(n).astype(np.float32))
    Ad = _dev_matrix(lib, A)
    for f in sorted({0, 1, min(n, 7), n // 2, n}):
        x_idx, xf = synth.frontier(n, f, seed=f + 3)
        mask = (rng.random(m) < 0.3).astype(np.uint8)
        for sched in range(12):
            _check(lib, A, Ad, semiring, x_idx, xf, None, True, sched)
        _check(lib, A, Ad, semiring, x_idx, xf, mask, True)
        _check(lib, A, Ad, semiring, x_idx, xf, mask, False)
    Ad.close()


@pytest.mark.parametrize("scale", [12, 16])
def test_rmat_frontier_sweep(lib, scale):
    A = synth.rmat(scale, seed=scale)
    Ad = _dev_matrix(lib, A)
    worst = 0.0
    for f in [1, 2, 100, 2047, 2048, 2049, 10000, A.n]:
        if f > A.n:
            continue
        x_idx, xf = synth.frontier(A.n, f, seed=f)
        for semiring in (0, 1, 2):
            for sched in (0, 1, 2, 3, 4, 5):
                worst = max(worst, _check(lib, A, Ad, semiring, x_idx, xf, None, True, sched))
    Ad.close()
    print("rmat s%d: worst |err|/sum|ax| = %.3g (bound %g)" % (scale, worst, FP_TOL))


def test_grid_frontiers(lib):
    A = synth.grid3d(40, 40, 40, 0.05, seed=3)
    Ad = _dev_matrix(lib, A)
    rng = np.random.default_rng(4)
    for f in [1, 300, 20000]:
        x_idx, xf = synth.frontier(A.n, f, seed=f)
        mask = (rng.random(A.m) < 0.5).astype(np.uint8)
        for semiring in (0, 1, 2):
            _check(lib, A, Ad, semiring, x_idx, xf)
            _check(lib, A, Ad, semiring, x_idx, xf, mask, True)
    Ad.close()


def test_unsorted_rows_and_pattern_matrix(lib):
    rng = np.random.default_rng(9)
    A = synth.erdos_renyi(3000, d=20, seed=2)
    for j in range(A.n):
        s, e = A.colptr[j], A.colptr[j + 1]
        A.rowidx[s:e] = rng.permutation(A.rowidx[s:e])
    Ad = _dev_matrix(lib, A)
    x_idx, xf = synth.frontier(A.n, 900, seed=1)
    for semiring in (0, 1, 2):
        _check(lib, A, Ad, semiring, x_idx, xf)
    Ad.close()
    P = synth.CSC(A.m, A.n, A.colptr, A.rowidx, None)
    Pd = _dev_matrix(lib, P)
    _check(lib, P, Pd, 0, x_idx, xf)
    Pd.close()


def test_edge_cases(lib):
    torch, S = lib
    A = synth.rmat(12, seed=1)
    Ad = _dev_matrix(lib, A)
    # empty x
    yi, yv, k, st = _run(lib, A, Ad, 0, np.zeros(0, np.int32), np.zeros(0, np.float32))
    assert k == 0 and st == 0
    # x selecting only empty columns
    iso = np.flatnonzero(np.diff(A.colptr) == 0).astype(np.int32)[:50]
    assert iso.shape[0] > 0
    yi, yv, k, st = _run(lib, A, Ad, 0, iso, np.ones(iso.shape[0], np.float32))
    assert k == 0 and st == 0
    assert S.spmspv_last_work(Ad.handle) == 0
    # every row masked out
    x_idx, xf = synth.frontier(A.n, 500, seed=5)
    _check(lib, A, Ad, 1, x_idx, xf, np.ones(A.m, np.uint8), True)
    # all of x: every non-empty column
    x_all = np.arange(A.n, dtype=np.int32)
    _check(lib, A, Ad, 0, x_all, np.ones(A.n, np.float32))
    Ad.close()


@pytest.mark.parametrize("semiring", [0, 1, 2])
def test_largest_row_count(lib, semiring):
    """m = 2^26, the most rows the 16-bit bucket offsets allow (8192 fine
    buckets of 8192 rows, 2048 buckets at the widest width): rows spread over
    the whole range, the first and the last row included; one more row is
    refused."""
    torch, S = lib
    m, n = 1 << 26, 2000
    rng = np.random.default_rng(26)
    cols = [np.unique(rng.integers(0, m, size=50)) for _ in range(n)]
    cols[0] = np.unique(np.concatenate([cols[0], [0, m - 1]]))
    cols[n - 1] = np.unique(np.concatenate([cols[n - 1], [m - 1, m - 2]]))
    colptr = np.concatenate([[0], np.cumsum([c.shape[0] for c in cols])]).astype(np.int32)
    rowidx = np.concatenate(cols).astype(np.int32)
    val = rng.random(rowidx.shape[0], dtype=np.float32)
    from types import SimpleNamespace
    A = SimpleNamespace(m=m, n=n, colptr=colptr, rowidx=rowidx, val=val, nnz=rowidx.shape[0])
    Ad = _dev_matrix(lib, A)
    x_all = np.arange(n, dtype=np.int32)
    _check(lib, A, Ad, semiring, x_all, rng.random(n, dtype=np.float32), sched=5)
    x_half = rng.permutation(n)[: n // 2].astype(np.int32)
    _check(lib, A, Ad, semiring, x_half, rng.random(x_half.shape[0], dtype=np.float32), sched=0)
    Ad.close()
    with pytest.raises(S.SpmspvError) as e:
        S.CscMatrix(m + 1, n, colptr, rowidx, val)
    assert e.value.code == S.SPMSPV_ERR_UNSUPPORTED


def test_capacity_overflow_reports_size_and_stays_in_bounds(lib):
    torch, S = lib
    A = synth.rmat(12, seed=1)
    Ad = _dev_matrix(lib, A)
    x_idx, xf = synth.frontier(A.n, 300, seed=2)
    ref = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, oracle.PLUS_TIMES, x_idx, xf)
    need = ref.idx.shape[0]
    cap = need // 2
    guard = 64
    y_idx = torch.full((cap + guard,), -7, dtype=torch.int32, device="cuda")
    y_val = torch.full((cap + guard,), -7.0, dtype=torch.float32, device="cuda")
    nnz = torch.zeros(1, dtype=torch.int32, device="cuda")
    xi = torch.from_numpy(x_idx).cuda()
    xv = torch.from_numpy(xf).cuda()
    S.spmspv_run(Ad.handle, 0, xi, xv, x_idx.shape[0], None, 0, y_idx, y_val, cap, nnz)
    assert int(nnz.item()) == need
    assert S.spmspv_device_status(Ad.handle) == S.SPMSPV_DEV_CAPACITY
    assert S.spmspv_device_status(Ad.handle) == 0  # reading clears it
    assert torch.all(y_idx[cap:] == -7) and torch.all(y_val[cap:] == -7.0)
    np.testing.assert_array_equal(y_idx[:cap].cpu().numpy(), ref.idx[:cap])
    Ad.close()


def test_bad_arguments_return_codes(lib):
    torch, S = lib
    A = synth.rmat(10, seed=1)
    Ad = _dev_matrix(lib, A)
    xi = torch.zeros(4, dtype=torch.int32, device="cuda")
    y = torch.zeros(A.m, dtype=torch.int32, device="cuda")
    nnz = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(S.SpmspvError) as e:
        S.spmspv_run(Ad.handle, 7, xi, None, 4, None, 0, y, None, A.m, nnz)
    assert e.value.code == S.SPMSPV_ERR_ARG
    with pytest.raises(S.SpmspvError) as e:
        S.spmspv_run(Ad.handle, 2, xi, None, A.n + 1, None, 0, y, None, A.m, nnz)
    assert e.value.code == S.SPMSPV_ERR_ARG
    with pytest.raises(S.SpmspvError) as e:
        S.spmspv_run(Ad.handle, 2, xi, None, 4, None, 0, y, None, A.m, None)
    assert e.value.code == S.SPMSPV_ERR_ARG
    with pytest.raises(S.SpmspvError) as e:
        S.spmspv_run(Ad.handle, 2, xi, None, 4, None, S.SPMSPV_SCHED_OPT(12), y, None, A.m, nnz)
    assert e.value.code == S.SPMSPV_ERR_ARG
    # an out-of-range x index is caught on the device, nothing is read out of bounds
    bad = torch.tensor([3, A.n + 5], dtype=torch.int32, device="cuda")
    S.spmspv_run(Ad.handle, 2, bad, None, 2, None, 0, y, None, A.m, nnz)
    assert S.spmspv_device_status(Ad.handle) & S.SPMSPV_DEV_INDEX
    # the handle still works afterwards
    x_idx, xf = synth.frontier(A.n, 100, seed=1)
    _check(lib, A, Ad, 0, x_idx, xf)
    Ad.close()
    # bad matrices
    cp = torch.tensor([0, 1], dtype=torch.int32, device="cuda")
    ri = torch.tensor([5], dtype=torch.int32, device="cuda")
    with pytest.raises(S.SpmspvError) as e:
        S.spmspv_create_csc(2, 1, 1, cp, ri, None, S.SPMSPV_VAL_NONE)
    assert e.value.code == S.SPMSPV_ERR_INDEX
    with pytest.raises(S.SpmspvError) as e:
        S.spmspv_create_csc(0, 1, 1, cp, ri, None, S.SPMSPV_VAL_NONE)
    assert e.value.code == S.SPMSPV_ERR_ARG


@pytest.mark.parametrize("tail", [0, 1, 2, 3])
def test_columns_at_the_end_of_the_arrays(lib, tail):
    # columns that end at the end of the arrays (nnz = 4k + tail), selected
    # alone and together with the first
    torch, S = lib
    rng = np.random.default_rng(tail)
    n, m = 37, 50
    deg = rng.integers(0, 9, size=n)
    deg[-1] = 5
    nnz = int(deg.sum())
    deg[-1] += (tail - nnz) % 4
    colptr = np.concatenate([[0], np.cumsum(deg)]).astype(np.int32)
    rowidx = np.concatenate([np.sort(rng.choice(m, size=d, replace=False)) for d in deg]).astype(np.int32)
    val = rng.random(rowidx.shape[0]).astype(np.float32)
    assert rowidx.shape[0] % 4 == tail
    Ad = S.CscMatrix(m, n, colptr, rowidx, val)
    for x_idx in (np.arange(n, dtype=np.int32), np.array([n - 1], np.int32), np.array([n - 1, 0], np.int32)):
        xf = rng.random(x_idx.shape[0]).astype(np.float32)
        for semiring in (0, 1, 2):
            xv = x_values(semiring, x_idx, xf)
            ref = oracle.spmspv(m, colptr, rowidx, val, SEMIRING_TO_ORACLE[semiring], x_idx, xv, None, True)
            yi, yv, k, st = _run(lib, None, Ad, semiring, x_idx, xv, None, True, None)
            assert st == 0
            compare(semiring, ref, yi, yv)
    Ad.close()


def test_many_calls_on_one_handle(lib):
    """Per-call device state (tickets, look-back words, bucket fills) resets itself."""
    A = synth.rmat(14, seed=7)
    Ad = _dev_matrix(lib, A)
    rng = np.random.default_rng(1)
    for it in range(40):
        f = int(rng.integers(0, A.n))
        semiring = int(rng.integers(0, 3))
        sched = int(rng.integers(0, 12))
        x_idx, xf = synth.frontier(A.n, f, seed=it)
        mask = (rng.random(A.m) < 0.2).astype(np.uint8) if it % 3 == 0 else None
        _check(lib, A, Ad, semiring, x_idx, xf, mask, True, sched)
    Ad.close()


@pytest.fixture(scope="module")
def rmat18(lib):
    return synth.rmat(18, seed=3)


@pytest.mark.parametrize("f", [2, 3, 1000, 65537, 200000])
@pytest.mark.parametrize("semiring", [0, 1, 2])
def test_presorted_x(lib, rmat18, f, semiring):
    """SPMSPV_SORT_X: x in random order is sorted on the device (a counting
    sort over 32 tiles of 8,192 ids here) before the product; y must equal the
    reference's, unmasked and masked, push and pull."""
    torch, S = lib
    A = rmat18
    Ad = _dev_matrix(lib, A, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
    x_idx, xf = synth.frontier(A.n, f, seed=f, stream=2)
    assert f < 3 or (np.diff(x_idx) < 0).any()  # really unsorted
    _check(lib, A, Ad, semiring, x_idx, xf, extra_opts=S.SPMSPV_SORT_X)
    mask = (np.random.default_rng(f).random(A.m) < 0.3).astype(np.uint8)
    _check(lib, A, Ad, semiring, x_idx, xf, mask, True, sched=2, extra_opts=S.SPMSPV_SORT_X)
    if semiring != 0:  # the pull form needs A == A^T with values for (+,*)
        _check(lib, A, Ad, semiring, x_idx, xf, mask, False, sched=8, extra_opts=S.SPMSPV_SORT_X)
    Ad.close()


def test_presort_flags_bad_ids(lib, rmat18):
    torch, S = lib
    A = rmat18
    Ad = _dev_matrix(lib, A)
    y = torch.empty(A.m, dtype=torch.int32, device="cuda")
    nnz = torch.zeros(1, dtype=torch.int32, device="cuda")
    bad = torch.tensor([3, A.n + 5, 17], dtype=torch.int32, device="cuda")
    S.spmspv_run(Ad.handle, 2, bad, None, 3, None, S.SPMSPV_SORT_X, y, None, A.m, nnz)
    assert S.spmspv_device_status(Ad.handle) & S.SPMSPV_DEV_INDEX
    # the bitmap was cleared behind the sort: the next sorted call is clean
    x_idx, xf = synth.frontier(A.n, 5000, seed=9)
    _check(lib, A, Ad, 0, x_idx, xf, extra_opts=S.SPMSPV_SORT_X)
    Ad.close()


@pytest.fixture(scope="module")
def rmat22(lib):
    return synth.rmat(22, seed=1)


@pytest.mark.parametrize("f", [100, 10000, 1000000])
def test_rmat22_full_size(lib, rmat22, f):
    """The R-MAT scale-22 sweep at its full size, every output checked."""
    A = rmat22
    Ad = _dev_matrix(lib, A)
    x_idx, xf = synth.frontier(A.n, f, seed=1, stream=2)
    w = _check(lib, A, Ad, 0, x_idx, xf)
    _check(lib, A, Ad, 1, x_idx, xf)
    print("rmat22 f=%d worst ratio %.3g" % (f, w))
    Ad.close()


def test_hub_rows_combined_per_tile(lib):
    """Rows with thousands of nonzeros take the hub path (combined per
    expand/scatter tile); results must not change."""
    rng = np.random.default_rng(12)
    n, m = 30000, 5000
    hubs = np.array([0, 17, 2500, 4999], np.int32)
    cols = []
    for j in range(n):
        r = rng.choice(m, size=int(rng.integers(0, 6)), replace=False).astype(np.int32)
        r = np.union1d(r, hubs[rng.random(hubs.shape[0]) < 0.8]).astype(np.int32)
        cols.append(r)
    colptr = np.zeros(n + 1, np.int32)
    colptr[1:] = np.cumsum([c.shape[0] for c in cols])
    rowidx = np.concatenate(cols).astype(np.int32)
    val = rng.random(rowidx.shape[0]).astype(np.float32)
    A = synth.CSC(m, n, colptr, rowidx, val)
    Ad = _dev_matrix(lib, A)
    for f in [1, 500, 8000, n]:
        x_idx, xf = synth.frontier(n, f, seed=f)
        mask = (rng.random(m) < 0.3).astype(np.uint8)
        mask[hubs[:2]] = 1
        for semiring in (0, 1, 2):
            for sched in (0, 4, 8):
                _check(lib, A, Ad, semiring, x_idx, xf, None, True, sched)
            _check(lib, A, Ad, semiring, x_idx, xf, mask, True)
            _check(lib, A, Ad, semiring, x_idx, xf, mask, False)
    Ad.close()


def test_unsorted_output_mode(lib):
    # the ER configuration in unsorted-output mode (no SPMSPV_SORTED_OUT): the
    # comparison sorts both sides (the library emits ascending rows anyway)
    torch, S = lib
    A = synth.erdos_renyi(65536, d=16, seed=1)
    Ad = _dev_matrix(lib, A)
    x_idx, xf = synth.frontier(A.n, 655, seed=1, stream=2)
    xi = torch.from_numpy(x_idx).cuda()
    yi, yv, k = Ad.multiply(0, xi, torch.from_numpy(xf).cuda(), None, 0)
    ref = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, SEMIRING_TO_ORACLE[0], x_idx, xf, None, True)
    yi_h, yv_h = yi.cpu().numpy()[:k], yv.cpu().numpy()[:k]
    order = np.argsort(yi_h, kind="stable")
    compare(0, ref, yi_h[order], yv_h[order])
    Ad.close()


def test_single_dense_column(lib):
    # one column holds every row (a product run far longer than a K2 tile)
    rng = np.random.default_rng(8)
    m, n = 20000, 12
    cols = [np.sort(rng.choice(m, size=rng.integers(0, 40), replace=False)) for _ in range(n)]
    cols[5] = np.arange(m)
    colptr = np.concatenate([[0], np.cumsum([c.shape[0] for c in cols])]).astype(np.int32)
    rowidx = np.concatenate(cols).astype(np.int32)
    val = rng.random(rowidx.shape[0]).astype(np.float32)
    from types import SimpleNamespace
    A = SimpleNamespace(m=m, n=n, colptr=colptr, rowidx=rowidx, val=val, nnz=rowidx.shape[0])
    Ad = _dev_matrix(lib, A)
    for x_idx in (np.array([5], np.int32), np.arange(n, dtype=np.int32), np.array([11, 5, 0], np.int32)):
        xf = rng.random(x_idx.shape[0]).astype(np.float32)
        for semiring in (0, 1, 2):
            _check(lib, A, Ad, semiring, x_idx, xf)
    Ad.close()


def test_bounded_wait_gives_up_and_reports(lib):
    # a look-back wait on a word nothing publishes runs out, records
    # SPMSPV_DEV_TIMEOUT and returns; the handle keeps giving exact results
    torch, S = lib
    A = synth.rmat(10, seed=2)
    Ad = _dev_matrix(lib, A)
    assert S.spmspv_device_status(Ad.handle) == 0
    S.spmspv_selftest_wait_timeout(Ad.handle, 2000)
    assert S.spmspv_device_status(Ad.handle) & S.SPMSPV_DEV_TIMEOUT
    assert S.spmspv_device_status(Ad.handle) == 0  # read and cleared
    x_idx, xf = synth.frontier(A.n, 200, seed=3)
    _check(lib, A, Ad, 0, x_idx, xf)
    with pytest.raises(S.SpmspvError):
        S.spmspv_selftest_wait_timeout(Ad.handle, 0)
    Ad.close()
