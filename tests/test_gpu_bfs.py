"""GPU BFS (device-side level loop) and the pull direction against the oracle.

Levels and parents must match the oracle bit for bit (Sec. IV-D level rule:
the parent is the smallest-id neighbour one level closer).  Every fixed
schedule is run: push (bucketed SpMSpV) and, for symmetric patterns, pull
(matrix-driven masked SpMV).
"""
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


GRAPHS = [
    ("rmat12", lambda: synth.rmat(12, seed=5), True),
    ("rmat14", lambda: synth.rmat(14, seed=6), True),
    ("grid3d", lambda: synth.grid3d(18, 17, 16, 0.05, seed=3), True),
    ("grid2d_long", lambda: synth.grid3d(300, 9, 1, 0.02, seed=3), True),
    ("er_directed", lambda: synth.erdos_renyi(5000, d=3, seed=9), False),
]


@pytest.mark.parametrize("name,make,sym", GRAPHS)
def test_bfs_all_fixed_schedules(lib, name, make, sym):
    torch, S = lib
    A = make()
    flags = S.SPMSPV_CSC_PATTERN_SYMMETRIC if sym else 0
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val, flags=flags)
    for src in synth.sources(A.colptr, 2, seed=3):
        ref_level, ref_parent, ref_nl, _, _ = oracle.bfs(A.colptr, A.rowidx, src)
        for sched in range(12):
            level, parent, nl = Ad.bfs(int(src), S.SPMSPV_SCHED_OPT(sched))
            assert S.spmspv_device_status(Ad.handle) == 0
            np.testing.assert_array_equal(level.cpu().numpy(), ref_level, err_msg="sched %d" % sched)
            np.testing.assert_array_equal(parent.cpu().numpy(), ref_parent, err_msg="sched %d" % sched)
            assert nl == ref_nl
        # default schedule, twice in a row on the same handle
        for _ in range(2):
            level, parent, nl = Ad.bfs(int(src))
            np.testing.assert_array_equal(level.cpu().numpy(), ref_level)
            assert nl == ref_nl
        # the direction-optimizing rule (push or pull per level by two thresholds;
        # push only without a pattern-symmetric handle)
        level, parent, nl = Ad.bfs(int(src), S.SPMSPV_SCHED_RULE)
        assert S.spmspv_device_status(Ad.handle) == 0
        np.testing.assert_array_equal(level.cpu().numpy(), ref_level, err_msg="rule")
        np.testing.assert_array_equal(parent.cpu().numpy(), ref_parent, err_msg="rule")
        assert nl == ref_nl
    Ad.close()


def test_direction_rule_switches_to_pull_and_back(lib):
    """On R-MAT the rule must take the pull direction for the wide middle levels
    and come back to push for the last ones; the result is the oracle's."""
    torch, S = lib
    A = synth.rmat(16, seed=8, values=False)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
    src = int(synth.sources(A.colptr, 1, seed=4)[0])
    rl, rp, nl_ref, _, sizes = oracle.bfs(A.colptr, A.rowidx, src)
    level, parent, nl = Ad.bfs(src, S.SPMSPV_SCHED_RULE)
    np.testing.assert_array_equal(level.cpu().numpy(), rl)
    np.testing.assert_array_equal(parent.cpu().numpy(), rp)
    assert nl == nl_ref and S.spmspv_device_status(Ad.handle) == 0
    # the rule's thresholds on the oracle's level sizes: some level is wide enough
    deg = np.diff(A.colptr).astype(np.int64)
    lv = rl
    seen, pulls = 0, 0
    for L in range(1, nl_ref):
        W = int(deg[lv == L - 1].sum())
        seen += W
        pulls += int(W * 14 > A.nnz - seen)
    assert pulls >= 1
    with pytest.raises(S.SpmspvError):
        Ad.bfs(src, S.SPMSPV_SCHED_RULE | S.SPMSPV_SCHED_AUTO)
    Ad.close()


def test_bfs_isolated_source_and_intact_grid(lib):
    torch, S = lib
    X, Y, Z = 11, 10, 9
    A = synth.grid3d(X, Y, Z, 0.0)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
    c = (5, 5, 4)
    src = c[0] * Y * Z + c[1] * Z + c[2]
    level, parent, nl = Ad.bfs(src)
    v = np.arange(A.n)
    x, y, z = v // (Y * Z), (v // Z) % Y, v % Z
    np.testing.assert_array_equal(level.cpu().numpy(),
                                  np.abs(x - c[0]) + np.abs(y - c[1]) + np.abs(z - c[2]))
    Ad.close()
    R = synth.rmat(11, seed=2)
    iso = int(np.flatnonzero(np.diff(R.colptr) == 0)[0])
    Rd = S.CscMatrix(R.m, R.n, R.colptr, R.rowidx, R.val, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
    level, parent, nl = Rd.bfs(iso)
    lv = level.cpu().numpy()
    assert nl == 1 and lv[iso] == 0 and (lv >= 0).sum() == 1
    Rd.close()


def symmetric_values(A):
    """Values with A(i,j) == A(j,i) on a pattern-symmetric matrix."""
    cols = np.repeat(np.arange(A.n, dtype=np.int64), np.diff(A.colptr))
    lo = np.minimum(cols, A.rowidx.astype(np.int64))
    hi = np.maximum(cols, A.rowidx.astype(np.int64))
    h = (lo * 0x9E3779B1 + hi * 0x85EBCA77) & 0xFFFFFF
    return (h.astype(np.float64) / float(1 << 24)).astype(np.float32)


@pytest.mark.parametrize("scale", [11, 14])
def test_pull_direction_all_semirings(lib, scale):
    torch, S = lib
    A = synth.rmat(scale, seed=scale)
    A.val = symmetric_values(A)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val, flags=S.SPMSPV_CSC_SYMMETRIC)
    rng = np.random.default_rng(scale)
    for f in [1, 300, A.n // 3, A.n]:
        x_idx, xf = synth.frontier(A.n, f, seed=f)
        mask = (rng.random(A.m) < 0.4).astype(np.uint8)
        for semiring in (0, 1, 2):
            xv = x_values(semiring, x_idx, xf)
            for msk, comp in ((None, True), (mask, True), (mask, False)):
                ref = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, SEMIRING_TO_ORACLE[semiring],
                                    x_idx, xv, msk, comp)
                for sched in (6, 10):  # pull schedules
                    from test_gpu_spmspv import _run
                    yi, yv, k, st = _run(lib, A, Ad, semiring, x_idx, xv, msk, comp, sched)
                    assert st == 0 and k == ref.idx.shape[0]
                    compare(semiring, ref, yi, yv)
    Ad.close()


@pytest.mark.parametrize("scale", [11, 14])
def test_pull_with_vertex_id_values_stops_early(lib, scale):
    # SPMSPV_X_IDS: (min, select2nd) with x(j) = j lets the pull stop at a
    # row's first frontier neighbour (the smallest, row ids ascending); the
    # result must equal the reference under masks, pull schedules and the
    # learned schedule, and a matrix whose columns are not sorted must still
    # give the minimum (no early stop there)
    torch, S = lib
    from paper_1610_07902_gb300 import selector
    A = synth.rmat(scale, seed=scale + 40, values=False)
    rng = np.random.default_rng(scale)
    perm_rows = A.rowidx.copy()
    for j in range(A.n):  # the same pattern with every column's row ids reversed
        a, b = A.colptr[j], A.colptr[j + 1]
        perm_rows[a:b] = perm_rows[a:b][::-1]
    for rows in (A.rowidx, perm_rows):
        Ad = S.CscMatrix(A.m, A.n, A.colptr, rows, None, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
        S.spmspv_selector_set(Ad.handle, selector.load()[0])
        for f in [1, 300, A.n // 3, A.n]:
            x_idx, _ = synth.frontier(A.n, f, seed=f)
            mask = (rng.random(A.m) < 0.4).astype(np.uint8)
            ref = oracle.spmspv(A.m, A.colptr, A.rowidx, None, oracle.MIN_SELECT2ND, x_idx, x_idx, mask, True)
            xd = torch.from_numpy(x_idx).cuda()
            md = torch.from_numpy(mask_bits(mask).view(np.int32)).cuda()
            for opts in (S.SPMSPV_SCHED_OPT(6), S.SPMSPV_SCHED_OPT(11), S.SPMSPV_SCHED_AUTO):
                yi, yv, k = Ad.multiply(1, xd, xd, md, opts | S.SPMSPV_MASK_COMPLEMENT | S.SPMSPV_X_IDS)
                assert k == ref.idx.shape[0]
                compare(1, ref, yi.cpu().numpy(), yv.cpu().numpy())
        assert S.spmspv_device_status(Ad.handle) == 0
        Ad.close()
