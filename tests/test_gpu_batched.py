"""Batched SpMSpV (concurrent lanes over a device-side frontier queue, and
the persistent one-launch form where noted) and
multi-source BFS against the oracle: every frontier's y must equal the
single-product result (index sets and integer values bit for bit, FP32 values
within the parity tolerance)."""
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


def make_batch(n, B, seed, fmax):
    rng = np.random.default_rng(seed)
    sizes = np.maximum(1, np.floor(10 ** rng.uniform(0, np.log10(fmax), B))).astype(np.int64)
    fronts = [synth.frontier(n, int(min(s, n)), seed=seed * 1000 + b) for b, s in enumerate(sizes)]
    return fronts


@pytest.mark.parametrize("lanes", [1, 3, 8])
@pytest.mark.parametrize("masked", [False, True])
def test_batched_matches_oracle(lib, lanes, masked):
    torch, S = lib
    A = synth.rmat(14, seed=4)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val)
    B = 40
    fronts = make_batch(A.n, B, 7 + lanes, 5000)
    words = (A.m + 31) // 32
    rng = np.random.default_rng(lanes)
    masks_u8 = [(rng.random(A.m) < 0.3).astype(np.uint8) for _ in range(B)]
    for semiring in (0, 1, 2):
        xs = [x_values(semiring, xi, xf) for xi, xf in fronts]
        x_cnt = np.array([xi.shape[0] for xi, _ in fronts], np.int32)
        x_off = np.concatenate([[0], np.cumsum(x_cnt)[:-1]]).astype(np.int32)
        x_idx = np.concatenate([xi for xi, _ in fronts]).astype(np.int32)
        y_cap = np.full(B, A.m, np.int32)
        y_off = (np.arange(B) * A.m).astype(np.int32)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        xv = None if semiring == 2 else dev(np.concatenate(xs))
        yi = torch.empty(B * A.m, dtype=torch.int32, device="cuda")
        yv = None if semiring == 2 else torch.empty(B * A.m, dtype=torch.float32 if semiring == 0 else torch.int32, device="cuda")
        nz = torch.zeros(B, dtype=torch.int32, device="cuda")
        msk = dev(np.concatenate([mask_bits(mm) for mm in masks_u8]).view(np.int32)) if masked else None
        opts = S.SPMSPV_MASK_COMPLEMENT if masked else 0
        S.spmspv_run_batched(Ad.handle, semiring, B, dev(x_off), dev(x_cnt), dev(x_idx), xv, msk,
                             words, opts, dev(y_off), dev(y_cap), yi, yv, nz, lanes)
        nz_h = nz.cpu().numpy()
        yi_h = yi.cpu().numpy()
        yv_h = None if yv is None else yv.cpu().numpy()
        for b in range(B):
            ref = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, SEMIRING_TO_ORACLE[semiring],
                                fronts[b][0], xs[b], masks_u8[b] if masked else None, True)
            assert nz_h[b] == ref.idx.shape[0], (semiring, b)
            o = y_off[b]
            compare(semiring, ref, yi_h[o:o + nz_h[b]], None if yv_h is None else yv_h[o:o + nz_h[b]])
        assert S.spmspv_device_status(Ad.handle) == 0
    Ad.close()


@pytest.mark.parametrize("form", ["lanes", "persistent"])
def test_multisource_bfs_matches_oracle(lib, form):
    torch, S = lib
    A = synth.rmat(12, seed=8)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
    srcs = synth.sources(A.colptr, 24, seed=4)
    B = srcs.shape[0]
    level = torch.empty(B * A.n, dtype=torch.int32, device="cuda")
    parent = torch.empty(B * A.n, dtype=torch.int32, device="cuda")
    nl = torch.zeros(1, dtype=torch.int32, device="cuda")
    lanes = 4 if form == "lanes" else S.SPMSPV_LANES_PERSISTENT
    S.spmspv_msbfs(Ad.handle, B, torch.from_numpy(srcs).cuda(), level, parent, nl, 0, lanes)
    lv = level.cpu().numpy().reshape(B, A.n)
    pa = parent.cpu().numpy().reshape(B, A.n)
    deepest = 0
    for b in range(B):
        rl, rp, rn, _, _ = oracle.bfs(A.colptr, A.rowidx, int(srcs[b]))
        np.testing.assert_array_equal(lv[b], rl)
        np.testing.assert_array_equal(pa[b], rp)
        deepest = max(deepest, rn)
    assert int(nl.item()) == deepest
    assert S.spmspv_device_status(Ad.handle) == 0
    Ad.close()


@pytest.mark.parametrize("schedule", [0, 2, 5])
def test_persistent_msbfs_grid_and_isolated_sources(lib, schedule):
    # a high-diameter grid (searches of different depths: some frontiers empty
    # while others run on), sources on isolated vertices (empty first
    # frontier) and a repeated source, every search against the reference
    torch, S = lib
    A = synth.grid3d(24, 20, 6, 0.1, seed=3, values=False)
    deg = np.diff(A.colptr)
    isolated = np.flatnonzero(deg == 0)
    srcs = synth.sources(A.colptr, 14, seed=11).astype(np.int32)
    extra = [int(isolated[0])] if isolated.size else []
    srcs = np.concatenate([srcs, np.array(extra + [int(srcs[0]), 0, A.n - 1], np.int32)])
    B = srcs.shape[0]
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None, flags=S.SPMSPV_CSC_SYMMETRIC)
    level = torch.empty(B * A.n, dtype=torch.int32, device="cuda")
    parent = torch.empty(B * A.n, dtype=torch.int32, device="cuda")
    nl = torch.zeros(1, dtype=torch.int32, device="cuda")
    S.spmspv_msbfs(Ad.handle, B, torch.from_numpy(srcs).cuda(), level, parent, nl,
                   S.SPMSPV_SCHED_OPT(schedule), S.SPMSPV_LANES_PERSISTENT)
    lv = level.cpu().numpy().reshape(B, A.n)
    pa = parent.cpu().numpy().reshape(B, A.n)
    deepest = 0
    for b in range(B):
        rl, rp, rn, _, _ = oracle.bfs(A.colptr, A.rowidx, int(srcs[b]))
        np.testing.assert_array_equal(lv[b], rl, err_msg="levels of source %d" % b)
        np.testing.assert_array_equal(pa[b], rp, err_msg="parents of source %d" % b)
        deepest = max(deepest, rn)
    assert deepest > 20 and int(nl.item()) == deepest
    assert S.spmspv_device_status(Ad.handle) == 0
    Ad.close()


def test_autotuned_batch_matches_and_caches(lib):
    torch, S = lib
    A = synth.rmat(13, seed=9)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val)
    B = 24
    fronts = make_batch(A.n, B, 31, 3000)
    x_cnt = np.array([xi.shape[0] for xi, _ in fronts], np.int32)
    x_off = np.concatenate([[0], np.cumsum(x_cnt)[:-1]]).astype(np.int32)
    x_idx = np.concatenate([xi for xi, _ in fronts]).astype(np.int32)
    x_val = np.concatenate([xf for _, xf in fronts]).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    y_cap = np.full(B, A.m, np.int32)
    y_off = (np.arange(B) * A.m).astype(np.int32)
    args = [dev(x_off), dev(x_cnt), dev(x_idx), dev(x_val)]
    outs = []
    for call in range(2):
        yi = torch.empty(B * A.m, dtype=torch.int32, device="cuda")
        yv = torch.empty(B * A.m, dtype=torch.float32, device="cuda")
        nz = torch.zeros(B, dtype=torch.int32, device="cuda")
        S.spmspv_run_batched(Ad.handle, 0, B, *args, None, 0, 0, dev(y_off), dev(y_cap), yi, yv, nz, 0)
        lanes, sched, cached = S.spmspv_last_tuned(Ad.handle)
        assert lanes in (0, 4, 16) and 0 <= sched < 6  # 0: the persistent form
        assert cached == (call == 1)
        outs.append((nz.cpu().numpy(), yi.cpu().numpy(), yv.cpu().numpy()))
    nz_h, yi_h, yv_h = outs[1]
    for b in range(B):
        ref = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, SEMIRING_TO_ORACLE[0], fronts[b][0],
                            fronts[b][1], None, True)
        o = y_off[b]
        assert nz_h[b] == ref.idx.shape[0]
        compare(0, ref, yi_h[o:o + nz_h[b]], yv_h[o:o + nz_h[b]])
    ent = S.spmspv_tune_entries(Ad.handle)
    assert len(ent) == 1 and ent[0][0] == S.spmspv_tune_key(0, 0, 0, B, int(x_cnt.sum()))
    assert ent[0][3] > 0
    # an override is used as given (lanes 3: the lanes form)
    S.spmspv_tune_set(Ad.handle, ent[0][0], 3, 5)
    S.spmspv_run_batched(Ad.handle, 0, B, *args, None, 0, 0, dev(y_off), dev(y_cap), yi, yv, nz, 0)
    assert S.spmspv_last_tuned(Ad.handle) == (3, 5, True)
    assert (nz.cpu().numpy() == nz_h).all()
    S.spmspv_tune_clear(Ad.handle)
    assert S.spmspv_tune_entries(Ad.handle) == []
    Ad.close()


def test_autotuned_msbfs_and_acl_match_fixed(lib):
    torch, S = lib
    A = synth.rmat(11, seed=12, values=False)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None, flags=S.SPMSPV_CSC_SYMMETRIC)
    srcs = torch.from_numpy(synth.sources(A.colptr, 16, seed=9).astype(np.int32)).cuda()
    B = srcs.shape[0]
    res = []
    for lanes in (4, 0):
        level = torch.empty(B * A.n, dtype=torch.int32, device="cuda")
        parent = torch.empty(B * A.n, dtype=torch.int32, device="cuda")
        S.spmspv_msbfs(Ad.handle, B, srcs, level, parent, None, 0, lanes)
        res.append((level.cpu().numpy(), parent.cpu().numpy()))
    assert (res[0][0] == res[1][0]).all() and (res[0][1] == res[1][1]).all()
    assert S.spmspv_last_tuned(Ad.handle)[2] is False
    p = torch.empty(B * A.n, dtype=torch.float32, device="cuda")
    r = torch.empty(B * A.n, dtype=torch.float32, device="cuda")
    S.spmspv_acl(Ad.handle, B, srcs, 0.15, 1e-5, 1000, p, r, None, 0)
    lanes, sched, cached = S.spmspv_last_tuned(Ad.handle)
    assert not cached and lanes in (0, 2, 4, 8, 16)  # 0: the persistent form
    P = p.cpu().numpy().reshape(B, A.n).astype(np.float64)
    R = r.cpu().numpy().reshape(B, A.n).astype(np.float64)
    assert np.abs(P.sum(1) + R.sum(1) - 1).max() < 1e-5
    assert len(S.spmspv_tune_entries(Ad.handle)) == 2
    Ad.close()


@pytest.mark.parametrize("bias", ["trained", "pull", "push"])
def test_learned_msbfs_matches_fixed(lib, bias):
    # the learned multi-source BFS picks push or pull per source and level in
    # the lanes; forcing pull everywhere (or push) through the output biases
    # of the network exercises both kernels; levels and parents never change
    torch, S = lib
    from oracle import mlp
    from paper_1610_07902_gb300 import selector
    params, _ = selector.load()
    params = params.copy()
    if bias == "pull":
        params[mlp.O_B3 + 6:mlp.O_B3 + 12] -= 1e4
    elif bias == "push":
        params[mlp.O_B3:mlp.O_B3 + 6] -= 1e4
    A = synth.rmat(12, seed=21, values=False)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
    S.spmspv_selector_set(Ad.handle, params)
    srcs = synth.sources(A.colptr, 20, seed=3).astype(np.int32)
    B = srcs.shape[0]
    ds = torch.from_numpy(srcs).cuda()
    out = []
    for opts, lanes in ((0, 4), (S.SPMSPV_SCHED_AUTO, 4), (S.SPMSPV_SCHED_AUTO, 0)):
        level = torch.empty(B * A.n, dtype=torch.int32, device="cuda")
        parent = torch.empty(B * A.n, dtype=torch.int32, device="cuda")
        S.spmspv_msbfs(Ad.handle, B, ds, level, parent, None, opts, lanes)
        out.append((level.cpu().numpy(), parent.cpu().numpy()))
    for lv, pa in out[1:]:
        np.testing.assert_array_equal(lv, out[0][0])
        np.testing.assert_array_equal(pa, out[0][1])
    for b in (0, B - 1):
        ref_l, ref_p, _, _, _ = oracle.bfs(A.colptr, A.rowidx, int(srcs[b]))
        np.testing.assert_array_equal(out[1][0][b * A.n:(b + 1) * A.n], ref_l)
        np.testing.assert_array_equal(out[1][1][b * A.n:(b + 1) * A.n], ref_p)
    assert S.spmspv_device_status(Ad.handle) == 0
    Ad.close()


@pytest.mark.parametrize("bias", ["trained", "pull", "push"])
def test_learned_persistent_msbfs_matches_oracle(lib, bias):
    # the persistent form with the learned schedule: per source and level the
    # network picks push (the batched launch) or pull (k_msbfs_pull); levels
    # of more than 2^21 products may pull, so the graph has several such
    # levels per search; forcing pull (or push) through the output biases
    # exercises both paths, every search against the reference
    torch, S = lib
    from oracle import mlp
    from paper_1610_07902_gb300 import selector
    params, _ = selector.load()
    params = params.copy()
    if bias == "pull":
        params[mlp.O_B3 + 6:mlp.O_B3 + 12] -= 1e4
    elif bias == "push":
        params[mlp.O_B3:mlp.O_B3 + 6] -= 1e4
    A = synth.rmat(17, seed=23, values=False)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
    S.spmspv_selector_set(Ad.handle, params)
    srcs = synth.sources(A.colptr, 12, seed=8).astype(np.int32)
    B = srcs.shape[0]
    level = torch.empty(B * A.n, dtype=torch.int32, device="cuda")
    parent = torch.empty(B * A.n, dtype=torch.int32, device="cuda")
    nl = torch.zeros(1, dtype=torch.int32, device="cuda")
    S.spmspv_msbfs(Ad.handle, B, torch.from_numpy(srcs).cuda(), level, parent, nl, S.SPMSPV_SCHED_AUTO,
                   S.SPMSPV_LANES_PERSISTENT)
    lv = level.cpu().numpy().reshape(B, A.n)
    pa = parent.cpu().numpy().reshape(B, A.n)
    deepest = 0
    for b in range(B):
        rl, rp, rn, _, _ = oracle.bfs(A.colptr, A.rowidx, int(srcs[b]))
        np.testing.assert_array_equal(lv[b], rl, err_msg="levels of source %d" % b)
        np.testing.assert_array_equal(pa[b], rp, err_msg="parents of source %d" % b)
        deepest = max(deepest, rn)
    assert int(nl.item()) == deepest
    assert S.spmspv_device_status(Ad.handle) == 0
    Ad.close()


def test_batched_edge_cases(lib):
    # empty frontiers among full ones, a single-frontier batch, and a frontier
    # whose y does not fit: it reports the size it needs, the others are exact
    torch, S = lib
    A = synth.rmat(11, seed=17)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    fronts = [synth.frontier(A.n, k, seed=40 + i) if k else (np.zeros(0, np.int32), np.zeros(0, np.float32))
              for i, k in enumerate([0, 50, 0, 300, 1, 0])]
    B = len(fronts)
    x_cnt = np.array([f[0].shape[0] for f in fronts], np.int32)
    x_off = np.concatenate([[0], np.cumsum(x_cnt)[:-1]]).astype(np.int32)
    x_idx = np.concatenate([f[0] for f in fronts] + [np.zeros(1, np.int32)]).astype(np.int32)
    x_val = np.concatenate([f[1] for f in fronts] + [np.zeros(1, np.float32)]).astype(np.float32)
    refs = [oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, SEMIRING_TO_ORACLE[0], f[0], f[1], None, True)
            for f in fronts]
    small = 3  # frontier 3's y needs far more
    assert refs[small].idx.shape[0] > 10
    y_cap = np.full(B, A.m, np.int32)
    y_cap[small] = 10
    y_off = (np.arange(B) * A.m).astype(np.int32)
    for lanes in (1, 4, S.SPMSPV_LANES_PERSISTENT):
        yi = torch.full((B * A.m,), -7, dtype=torch.int32, device="cuda")
        yv = torch.zeros(B * A.m, dtype=torch.float32, device="cuda")
        nz = torch.full((B,), -1, dtype=torch.int32, device="cuda")
        S.spmspv_run_batched(Ad.handle, 0, B, dev(x_off), dev(x_cnt), dev(x_idx), dev(x_val), None, 0, 0,
                             dev(y_off), dev(y_cap), yi, yv, nz, lanes)
        nz_h, yi_h, yv_h = nz.cpu().numpy(), yi.cpu().numpy(), yv.cpu().numpy()
        for b in range(B):
            assert nz_h[b] == refs[b].idx.shape[0], (lanes, b)
            o = y_off[b]
            if b == small:
                np.testing.assert_array_equal(yi_h[o:o + 10], refs[b].idx[:10])
                assert (yi_h[o + 10:o + 20] == -7).all()  # nothing past the capacity
            else:
                compare(0, refs[b], yi_h[o:o + nz_h[b]], yv_h[o:o + nz_h[b]])
        assert S.spmspv_device_status(Ad.handle) & S.SPMSPV_DEV_CAPACITY
    # one frontier
    yi = torch.empty(A.m, dtype=torch.int32, device="cuda")
    yv = torch.empty(A.m, dtype=torch.float32, device="cuda")
    nz = torch.zeros(1, dtype=torch.int32, device="cuda")
    S.spmspv_run_batched(Ad.handle, 0, 1, dev(np.zeros(1, np.int32)), dev(x_cnt[3:4]), dev(fronts[3][0]),
                         dev(fronts[3][1]), None, 0, 0, dev(np.zeros(1, np.int32)),
                         dev(np.array([A.m], np.int32)), yi, yv, nz, 2)
    k = int(nz.item())
    compare(0, refs[3], yi.cpu().numpy()[:k], yv.cpu().numpy()[:k])
    Ad.close()
