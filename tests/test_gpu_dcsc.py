"""DCSC matrices on the GPU (only the columns holding entries stored, found
through the auxiliary column index) against the reference run on the same
matrix in CSC form: y bit for bit (values within the FP32 bound for (+,*)) on
a hypersparse rectangular matrix with x naming stored and unstored columns,
every semiring, masks, every push schedule, the device presort; and BFS,
connected components, independent sets and matching on a square graph with
isolated vertices stored as DCSC."""
from types import SimpleNamespace

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


def to_dcsc(colptr):
    """Stored columns (ids, ascending) and their pointers from CSC pointers."""
    deg = np.diff(colptr)
    jc = np.flatnonzero(deg > 0).astype(np.int32)
    cp = np.concatenate([[0], np.cumsum(deg[jc])]).astype(np.int32)
    return jc, cp


def hypersparse(m, n, nzc, seed):
    """m-by-n with nzc stored columns of 1..40 entries (three long ones)."""
    rng = np.random.default_rng(seed)
    cols = np.sort(rng.choice(n, size=nzc, replace=False)).astype(np.int64)
    d = rng.integers(1, 41, size=nzc)
    d[:3] = [600, 1, 2000]
    key = np.unique(np.repeat(cols, d) * m + rng.integers(0, m, size=int(d.sum())))
    col, row = key // m, key % m
    deg = np.bincount(col, minlength=n)
    colptr = np.concatenate([[0], np.cumsum(deg)]).astype(np.int32)
    val = rng.random(key.shape[0], dtype=np.float32) + 0.01
    return SimpleNamespace(m=m, n=n, colptr=colptr, rowidx=row.astype(np.int32), val=val,
                           nnz=key.shape[0], cols=cols.astype(np.int32))


@pytest.fixture(scope="module")
def hyper():
    return hypersparse(60000, 3_000_000, 20000, 11)


def _x(A, seed, stored, unstored):
    rng = np.random.default_rng(seed)
    a = rng.choice(A.cols, size=stored, replace=False)
    others = np.setdiff1d(rng.choice(A.n, size=unstored * 2, replace=False), A.cols)[:unstored]
    idx = rng.permutation(np.concatenate([a, others])).astype(np.int32)
    return idx, rng.random(idx.shape[0], dtype=np.float32)


@pytest.mark.parametrize("semiring", [0, 1, 2])
@pytest.mark.parametrize("sched", [0, 2, 3, 5])
def test_dcsc_spmspv_matches_reference(lib, hyper, semiring, sched):
    torch, S = lib
    A = hyper
    jc, cp = to_dcsc(A.colptr)
    assert jc.shape[0] == 20000
    Ad = S.DcscMatrix(A.m, A.n, jc, cp, A.rowidx, A.val)
    for seed, stored, unstored in ((1, 3000, 3000), (2, 20000, 500), (3, 0, 50), (4, 1, 0)):
        x_idx, xf = _x(A, seed + 10 * sched, stored, unstored)
        xv = x_values(semiring, x_idx, xf)
        mask = None
        if seed == 2:
            mask = (np.random.default_rng(seed).random(A.m) < 0.5).astype(np.uint8)
        ref = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, SEMIRING_TO_ORACLE[semiring], x_idx, xv,
                            mask, True)
        xi = torch.from_numpy(x_idx).cuda()
        xvd = None if xv is None else torch.from_numpy(xv).cuda()
        md = None if mask is None else torch.from_numpy(mask_bits(mask).view(np.int32)).cuda()
        for extra in (0, S.SPMSPV_SORT_X):
            opts = S.SPMSPV_SORTED_OUT | S.SPMSPV_SCHED_OPT(sched) | extra
            if md is not None:
                opts |= S.SPMSPV_MASK_COMPLEMENT
            yi, yv, k = Ad.multiply(semiring, xi, xvd, md, opts)
            assert S.spmspv_device_status(Ad.handle) == 0
            assert k == ref.idx.shape[0]
            compare(semiring, ref, yi.cpu().numpy(), None if yv is None else yv.cpu().numpy())
            assert S.spmspv_last_work(Ad.handle) == ref.nmult
    Ad.close()


def test_dcsc_without_stored_columns(lib):
    torch, S = lib
    Ad = S.DcscMatrix(100, 5000, np.zeros(0, np.int32), np.zeros(1, np.int32), np.zeros(0, np.int32))
    xi = torch.tensor([0, 17, 4999], dtype=torch.int32, device="cuda")
    yi, yv, k = Ad.multiply(2, xi)
    assert k == 0 and S.spmspv_device_status(Ad.handle) == 0
    Ad.close()


def test_dcsc_rejects_bad_arrays(lib):
    torch, S = lib
    rows = np.array([0, 1, 2], np.int32)
    for jc, cp in (([3, 1], [0, 1, 3]),      # not ascending
                   ([1, 9], [0, 1, 3]),      # id outside [0, n)
                   ([1, 3], [0, 2, 1]),      # pointers decrease
                   ([1, 3], [0, 1, 2])):     # pointers do not end at nnz
        with pytest.raises(S.SpmspvError):
            S.DcscMatrix(4, 5, np.array(jc, np.int32), np.array(cp, np.int32), rows)


@pytest.fixture(scope="module")
def graph():
    # R-MAT s14 has isolated vertices: their columns are the ones DCSC drops
    A = synth.rmat(14, seed=21, values=False)
    jc, cp = to_dcsc(A.colptr)
    assert jc.shape[0] < A.n
    return A, jc, cp


def test_dcsc_graph_algorithms(lib, graph):
    torch, S = lib
    A, jc, cp = graph
    flags = S.SPMSPV_CSC_PATTERN_SYMMETRIC
    Ad = S.DcscMatrix(A.m, A.n, jc, cp, A.rowidx, None, flags=flags)
    src = int(jc[7])
    for opts in (S.SPMSPV_SCHED_OPT(5), S.SPMSPV_SCHED_OPT(1)):
        level, parent, nl = Ad.bfs(src, opts)
        rl, rp = oracle.bfs(A.colptr, A.rowidx, src)[:2]
        np.testing.assert_array_equal(level.cpu().numpy(), rl)
        np.testing.assert_array_equal(parent.cpu().numpy(), rp)
    labels = torch.empty(A.n, dtype=torch.int32, device="cuda")
    S.spmspv_cc(Ad.handle, labels)
    np.testing.assert_array_equal(labels.cpu().numpy(), oracle.cc(A.colptr, A.rowidx)[0])
    prio = np.random.default_rng(5).permutation(A.n).astype(np.int32)
    in_set = torch.empty(A.n, dtype=torch.int32, device="cuda")
    S.spmspv_mis(Ad.handle, torch.from_numpy(prio).cuda(), in_set)
    np.testing.assert_array_equal(in_set.cpu().numpy(), oracle.mis(A.colptr, A.rowidx, prio)[0])
    mate_r = torch.empty(A.m, dtype=torch.int32, device="cuda")
    mate_c = torch.empty(A.n, dtype=torch.int32, device="cuda")
    card = torch.zeros(1, dtype=torch.int32, device="cuda")
    S.spmspv_mcm(Ad.handle, mate_r, mate_c, card)
    assert int(card.item()) == oracle.mcm(A.m, A.colptr, A.rowidx)[2]
    assert S.spmspv_device_status(Ad.handle) == 0
    # a pull schedule runs as its push form (no CSR view of a DCSC matrix)
    x_idx = jc[:300].copy()
    yi, yv, k = Ad.multiply(1, torch.from_numpy(x_idx).cuda(), torch.from_numpy(x_idx).cuda(), None,
                            S.SPMSPV_SORTED_OUT | S.SPMSPV_SCHED_OPT(8))
    ref = oracle.spmspv(A.m, A.colptr, A.rowidx, None, oracle.MIN_SELECT2ND, x_idx, x_idx, None, True)
    compare(1, ref, yi.cpu().numpy(), yv.cpu().numpy())
    # ACL reads degrees from CSC column pointers
    with pytest.raises(S.SpmspvError) as e:
        seeds = torch.tensor([src], dtype=torch.int32, device="cuda")
        p = torch.empty(A.n, dtype=torch.float32, device="cuda")
        r = torch.empty(A.n, dtype=torch.float32, device="cuda")
        S.spmspv_acl(Ad.handle, 1, seeds, 0.15, 1e-6, 10, p, r, None, 1)
    assert e.value.code == S.SPMSPV_ERR_UNSUPPORTED
    Ad.close()


def test_dcsc_learned_schedule(lib, graph):
    """The learned selector on a DCSC handle: push schedules only (no CSR view),
    same results as the reference for a plain product and a BFS."""
    torch, S = lib
    from paper_1610_07902_gb300 import selector
    try:
        params = selector.load()[0]
    except (OSError, ValueError, KeyError):
        pytest.skip("no selector weights")
    A, jc, cp = graph
    Ad = S.DcscMatrix(A.m, A.n, jc, cp, A.rowidx, None, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
    S.spmspv_selector_set(Ad.handle, params)
    x_idx = np.random.default_rng(3).permutation(jc)[:2000].astype(np.int32)
    xd = torch.from_numpy(x_idx).cuda()
    yi, yv, k = Ad.multiply(1, xd, xd, None, S.SPMSPV_SORTED_OUT | S.SPMSPV_SCHED_AUTO)
    ref = oracle.spmspv(A.m, A.colptr, A.rowidx, None, oracle.MIN_SELECT2ND, x_idx, x_idx, None, True)
    compare(1, ref, yi.cpu().numpy(), yv.cpu().numpy())
    assert S.spmspv_last_schedule(Ad.handle) < 6  # a push schedule
    src = int(jc[11])
    level, parent, nl = Ad.bfs(src, S.SPMSPV_SCHED_AUTO)
    rl, rp = oracle.bfs(A.colptr, A.rowidx, src)[:2]
    np.testing.assert_array_equal(level.cpu().numpy(), rl)
    np.testing.assert_array_equal(parent.cpu().numpy(), rp)
    assert S.spmspv_device_status(Ad.handle) == 0
    Ad.close()


def test_dcsc_batched_multi_source_bfs(lib, graph):
    torch, S = lib
    A, jc, cp = graph
    Ad = S.DcscMatrix(A.m, A.n, jc, cp, A.rowidx, None, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
    srcs = jc[np.random.default_rng(2).choice(jc.shape[0], size=6, replace=False)].astype(np.int32)
    B = srcs.shape[0]
    level = torch.empty(B * A.n, dtype=torch.int32, device="cuda")
    parent = torch.empty(B * A.n, dtype=torch.int32, device="cuda")
    nl = torch.zeros(B, dtype=torch.int32, device="cuda")
    S.spmspv_msbfs(Ad.handle, B, torch.from_numpy(srcs).cuda(), level, parent, nl, S.SPMSPV_SCHED_OPT(5), 2)
    lv = level.cpu().numpy().reshape(B, A.n)
    pv = parent.cpu().numpy().reshape(B, A.n)
    for b in range(B):
        rl, rp = oracle.bfs(A.colptr, A.rowidx, int(srcs[b]))[:2]
        np.testing.assert_array_equal(lv[b], rl)
        np.testing.assert_array_equal(pv[b], rp)
    assert S.spmspv_device_status(Ad.handle) == 0
    Ad.close()
