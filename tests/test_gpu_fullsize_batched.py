"""The batched workloads at the size the benchmark times them (R-MAT s20, 256
frontiers / sources / seeds, autotuned lanes and schedules as in the bench)
against the reference: every one of the 256 batched products checked element
by element; the multi-source BFS (autotuned, learned schedule and the
persistent form) from all 256 sources level for level and parent for parent;
ACL element by element on a sample of seeds (the reference is FP64 and the
device decides its pushing sets in FP32), with the properties every seed must
satisfy checked for all of them."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import acl_compare, compare, need_gpu

pytestmark = pytest.mark.gpu
B = 256


@pytest.fixture(scope="module")
def lib():
    torch = need_gpu()
    from paper_1610_07902_gb300 import spmspv as S
    S.load()
    return torch, S


@pytest.fixture(scope="module")
def rmat20():
    return synth.rmat(20, 16, seed=4)


def test_batched_spmspv_full_size(lib, rmat20):
    torch, S = lib
    A = rmat20
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val)
    rng = np.random.default_rng(4)
    sizes = np.maximum(1, np.floor(10 ** rng.uniform(0, 5, B))).astype(np.int64)
    fronts = [synth.frontier(A.n, int(f), seed=100 + b, stream=2) for b, f in enumerate(sizes)]
    x_cnt = sizes.astype(np.int32)
    x_off = np.concatenate([[0], np.cumsum(x_cnt)[:-1]]).astype(np.int32)
    td = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ycap = A.m
    yi = torch.empty(B * ycap, dtype=torch.int32, device="cuda")
    yv = torch.empty(B * ycap, dtype=torch.float32, device="cuda")
    nz = torch.zeros(B, dtype=torch.int32, device="cuda")
    y_off = (np.arange(B, dtype=np.int64) * ycap).astype(np.int32)
    S.spmspv_run_batched(Ad.handle, S.SPMSPV_PLUS_TIMES_F32, B, td(x_off), td(x_cnt),
                         td(np.concatenate([f[0] for f in fronts])), td(np.concatenate([f[1] for f in fronts])),
                         None, 0, 0, td(y_off), td(np.full(B, ycap, np.int32)), yi, yv, nz, 0)
    assert S.spmspv_device_status(Ad.handle) == 0
    nz_h, yi_h, yv_h = nz.cpu().numpy(), yi.cpu().numpy(), yv.cpu().numpy()
    for b in range(B):
        ref = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, oracle.PLUS_TIMES, fronts[b][0], fronts[b][1])
        o, k = int(y_off[b]), int(nz_h[b])
        assert k == ref.idx.shape[0], b
        compare(0, ref, yi_h[o:o + k], yv_h[o:o + k])
    Ad.close()


@pytest.fixture(scope="module")
def pattern20(lib, rmat20):
    torch, S = lib
    A = rmat20
    Ap = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None, flags=S.SPMSPV_CSC_SYMMETRIC)
    srcs = synth.sources(A.colptr, B, seed=5).astype(np.int32)
    yield A, Ap, srcs
    Ap.close()


@pytest.fixture(scope="module")
def bfs_refs20(pattern20):
    from test_gpu_fullsize_bfs import oracle_bfs_all
    A, _, srcs = pattern20
    return oracle_bfs_all(A, srcs)


@pytest.mark.parametrize("form", ["tuned", "learned", "persistent"])
def test_msbfs_full_size(lib, pattern20, bfs_refs20, form):
    torch, S = lib
    A, Ap, srcs = pattern20
    opts = 0
    lanes = S.SPMSPV_LANES_PERSISTENT if form == "persistent" else 0
    if form == "learned":
        from paper_1610_07902_gb300 import selector
        try:
            params = selector.load()[0]
        except (OSError, ValueError, KeyError):
            pytest.skip("no selector weights")
        S.spmspv_selector_set(Ap.handle, params)
        opts = S.SPMSPV_SCHED_AUTO
    lv = torch.empty(B * A.n, dtype=torch.int32, device="cuda")
    pa = torch.empty(B * A.n, dtype=torch.int32, device="cuda")
    S.spmspv_msbfs(Ap.handle, B, torch.from_numpy(srcs).cuda(), lv, pa, None, opts, lanes)
    assert S.spmspv_device_status(Ap.handle) == 0
    L = lv.view(B, A.n)
    P = pa.view(B, A.n)
    # every source against the reference (levels are unique and the parent is
    # the smallest-id neighbour one level up, so both are compared bit for bit)
    refs = bfs_refs20
    lv_h, pa_h = lv.cpu().numpy().reshape(B, A.n), pa.cpu().numpy().reshape(B, A.n)
    for b in range(B):
        rl, rp, _ = refs[b]
        np.testing.assert_array_equal(lv_h[b], rl, err_msg="levels of source %d" % b)
        np.testing.assert_array_equal(pa_h[b], rp, err_msg="parents of source %d" % b)
    # and, independently of the reference, the properties that single out that
    # answer: the parent of every reached vertex is a neighbour at level - 1,
    # and no neighbour at level - 1 has a smaller id
    rows = torch.from_numpy(A.rowidx.astype(np.int64)).cuda()
    cols = torch.repeat_interleave(torch.arange(A.n, device="cuda"),
                                   torch.from_numpy(np.diff(A.colptr).astype(np.int64)).cuda())
    key_edges = torch.sort(cols * A.n + rows).values
    big = torch.iinfo(torch.int64).max
    for b in range(0, B, 8):
        l, p = L[b].long(), P[b].long()
        assert int(l[int(srcs[b])]) == 0 and int(p[int(srcs[b])]) == int(srcs[b])
        reached = (l > 0).nonzero().flatten()
        assert bool((l[p[reached]] == l[reached] - 1).all()), b
        key = p[reached] * A.n + reached  # edge (parent -> v) stored in column parent
        pos = torch.searchsorted(key_edges, key).clamp(max=key_edges.numel() - 1)
        assert bool((key_edges[pos] == key).all()), b
        up = (l[cols] >= 0) & (l[cols] == l[rows] - 1)
        best = torch.full((A.n,), big, dtype=torch.int64, device="cuda").scatter_reduce(
            0, rows, torch.where(up, cols, torch.full_like(cols, big)), "amin")
        assert bool((best[reached] == p[reached]).all()), b


def test_acl_full_size(lib, pattern20):
    torch, S = lib
    A, Ap, srcs = pattern20
    alpha, eps = 0.15, 1e-6
    p = torch.empty(B * A.n, dtype=torch.float32, device="cuda")
    r = torch.empty(B * A.n, dtype=torch.float32, device="cuda")
    S.spmspv_acl(Ap.handle, B, torch.from_numpy(srcs).cuda(), alpha, eps, 100000, p, r, None, 0)
    assert S.spmspv_device_status(Ap.handle) == 0
    Pm, Rm = p.view(B, A.n).double(), r.view(B, A.n).double()
    assert float((Pm.sum(1) + Rm.sum(1) - 1).abs().max()) < 1e-5
    assert bool((Pm >= 0).all() and (Rm >= 0).all())
    deg = torch.from_numpy(np.diff(A.colptr).astype(np.float64)).cuda()
    assert bool(((Rm < eps * deg * (1 + 1e-4)) | ((deg == 0) & (Rm == 0))).all())
    P_h, R_h = Pm.cpu().numpy(), Rm.cpu().numpy()
    # element by element against the FP64 trace on a sample of 32 seeds (a
    # few seconds each on the host, run in a thread pool)
    from concurrent.futures import ThreadPoolExecutor
    import os
    sample = np.random.default_rng(7).choice(B, size=32, replace=False)
    with ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1))) as ex:
        out = list(ex.map(lambda b: acl_compare(P_h[b], R_h[b], A.colptr, A.rowidx, int(srcs[b]),
                                                alpha, eps, 100000), sample))
    print("ACL s20: seeds with near-threshold vertices %d of %d, disagreeing vertices %d" % (
        sum(1 for nr, _ in out if nr), len(out), sum(d for _, d in out)))
