"""The direct (+,*) form (products added into a dense accumulator in device
memory, touched rows read back in order and reset) against the oracle: on
both sides of its threshold (2m products), with hub rows, masks, a y that is
too small, repeated calls (the accumulator must be clean after every call),
a DCSC handle and the learned schedule."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import compare, mask_bits, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = need_gpu()
    from paper_1610_07902_gb300 import spmspv as S
    S.load()
    return torch, S


def run(torch, S, Ad, A, xi, xf, opts=0, mask_u8=None, complement=True, cap=None):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    mask = None
    if mask_u8 is not None:
        mask = t(mask_bits(mask_u8).view(np.int32))
        if complement:
            opts |= S.SPMSPV_MASK_COMPLEMENT
    yi, yv, k = Ad.multiply(0, t(xi), t(xf), mask, opts, y_capacity=cap)
    ref = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, oracle.PLUS_TIMES, xi, xf, mask_u8, complement)
    st = S.spmspv_device_status(Ad.handle)
    return yi.cpu().numpy(), yv.cpu().numpy(), k, ref, st


def test_direct_both_sides_of_the_threshold_and_repeats(lib):
    torch, S = lib
    A = synth.rmat(16, seed=13)   # hub rows (relabelled) among the others
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val)
    deg = np.diff(A.colptr)
    rng = np.random.default_rng(3)
    order = rng.permutation(A.n)
    # frontiers whose products sit just below and above 2m, then others
    cum = np.cumsum(deg[order])
    thr = int(np.searchsorted(cum, 2 * A.m))
    sizes = [thr - 2, thr + 2, 3000, 20000, 64]
    for f in sizes:
        xi = np.sort(order[:f]).astype(np.int32)
        xf = rng.uniform(-1, 1, f).astype(np.float32)
        for opts in (0, S.SPMSPV_BUCKETS_ONLY, S.SPMSPV_SCHED_OPT(0), S.SPMSPV_SCHED_OPT(3)):
            yi, yv, k, ref, st = run(torch, S, Ad, A, xi, xf, opts)
            assert st == 0 and k == ref.idx.shape[0], (f, opts)
            compare(0, ref, yi, yv)
        order = np.roll(order, 977)
    Ad.close()


def test_direct_masks_capacity_and_recovery(lib):
    torch, S = lib
    A = synth.rmat(15, seed=17)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val)
    rng = np.random.default_rng(9)
    xi, xf = synth.frontier(A.n, 8000, seed=5)
    mask = (rng.random(A.m) < 0.4).astype(np.uint8)
    for comp in (True, False):
        yi, yv, k, ref, st = run(torch, S, Ad, A, xi, xf, 0, mask, comp)
        assert st == 0 and k == ref.idx.shape[0]
        compare(0, ref, yi, yv)
    # y too small: the size needed is reported, the first entries are right,
    # and the accumulator is clean for the next call
    yi, yv, k, ref, st = run(torch, S, Ad, A, xi, xf, 0, cap=100)
    assert st == S.SPMSPV_DEV_CAPACITY and k == ref.idx.shape[0] and k > 100
    np.testing.assert_array_equal(yi[:100], ref.idx[:100])
    for seed in range(3):
        xi2, xf2 = synth.frontier(A.n, 6000 + 1000 * seed, seed=20 + seed)
        yi, yv, k, ref, st = run(torch, S, Ad, A, xi2, xf2)
        assert st == 0 and k == ref.idx.shape[0]
        compare(0, ref, yi, yv)
    Ad.close()


def test_direct_on_dcsc_and_learned(lib):
    torch, S = lib
    from paper_1610_07902_gb300 import selector
    A = synth.rmat(14, seed=19)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    deg = np.diff(A.colptr)
    jc = np.nonzero(deg)[0].astype(np.int32)
    cp = np.concatenate([[0], np.cumsum(deg[jc])]).astype(np.int32)
    h = S.spmspv_create_dcsc(A.m, A.n, A.nnz, jc.shape[0], t(jc), t(cp), t(A.rowidx), t(A.val))
    xi, xf = synth.frontier(A.n, 4000, seed=8)
    ref = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, oracle.PLUS_TIMES, xi, xf)
    yi = torch.empty(A.m, dtype=torch.int32, device="cuda")
    yv = torch.empty(A.m, dtype=torch.float32, device="cuda")
    nz = torch.zeros(1, dtype=torch.int32, device="cuda")
    S.spmspv_run(h, 0, t(xi), t(xf), xi.shape[0], None, 0, yi, yv, A.m, nz)
    k = int(nz.item())
    assert S.spmspv_device_status(h) == 0 and k == ref.idx.shape[0]
    compare(0, ref, yi.cpu().numpy()[:k], yv.cpu().numpy()[:k])
    S.spmspv_destroy(h)
    # (pattern-symmetric: the values are not, so (+,*) stays push)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
    S.spmspv_selector_set(Ad.handle, selector.load()[0])
    for f in (100, 4000):
        xi, xf = synth.frontier(A.n, f, seed=f)
        yi, yv, k, ref, st = run(torch, S, Ad, A, xi, xf, S.SPMSPV_SCHED_AUTO)
        assert st == 0 and k == ref.idx.shape[0]
        compare(0, ref, yi, yv)
    Ad.close()
