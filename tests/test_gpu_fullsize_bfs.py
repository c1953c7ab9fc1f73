"""BFS and a masked product at the benchmark's sizes against the reference:
R-MAT s22 from all 64 sources the benchmark times, under the fixed schedule
and the learned one, the 256^3 grid from its centre (385 levels), and a
complemented-mask (select2nd, min) product with 10^6 x entries on R-MAT s22 —
every output compared element by element.  The reference searches run in a
thread pool (the oracle's C code releases the interpreter lock)."""
from concurrent.futures import ThreadPoolExecutor
import os

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


@pytest.fixture(scope="module")
def rmat22():
    return synth.rmat(22, seed=1)


def oracle_bfs_all(A, srcs):
    """The reference BFS of every source, computed in a thread pool."""
    threads = max(1, min(16, os.cpu_count() or 1))
    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(lambda s: oracle.bfs(A.colptr, A.rowidx, int(s))[:3], srcs))


def _bfs_check(torch, S, A, srcs, opts_list, params=None):
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
    if params is not None:
        S.spmspv_selector_set(Ad.handle, params)
    refs = oracle_bfs_all(A, srcs)
    for src, (rl, rp, nl_ref) in zip(srcs, refs):
        for opts in opts_list:
            level, parent, nl = Ad.bfs(int(src), opts)
            np.testing.assert_array_equal(level.cpu().numpy(), rl)
            np.testing.assert_array_equal(parent.cpu().numpy(), rp)
            assert nl == nl_ref
    assert S.spmspv_device_status(Ad.handle) == 0
    Ad.close()


def test_bfs_rmat22_fixed_and_learned(lib, rmat22):
    torch, S = lib
    from paper_1610_07902_gb300 import selector
    try:
        params = selector.load()[0]
        opts = [S.SPMSPV_SCHED_OPT(5), S.SPMSPV_SCHED_AUTO]
    except (OSError, ValueError, KeyError):
        params, opts = None, [S.SPMSPV_SCHED_OPT(5)]
    srcs = synth.sources(rmat22.colptr, 64, seed=2)  # every source the benchmark times
    _bfs_check(torch, S, rmat22, srcs, opts, params)


def test_bfs_grid256_from_centre(lib):
    torch, S = lib
    G = synth.grid3d(256, 256, 256, 0.05, seed=3, values=False)
    _bfs_check(torch, S, G, [128 * 65536 + 128 * 256 + 128], [S.SPMSPV_SCHED_OPT(5), S.SPMSPV_SCHED_OPT(2)])


def test_masked_min_product_rmat22(lib, rmat22):
    torch, S = lib
    A = rmat22
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val)
    x_idx, _ = synth.frontier(A.n, 1_000_000, seed=1, stream=2)
    mask = (np.random.default_rng(22).random(A.m) < 0.4).astype(np.uint8)
    ref = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, oracle.MIN_SELECT2ND, x_idx, x_idx, mask, True)
    xd = torch.from_numpy(x_idx).cuda()
    md = torch.from_numpy(mask_bits(mask).view(np.int32)).cuda()
    yi, yv, k = Ad.multiply(1, xd, xd, md, S.SPMSPV_SORTED_OUT | S.SPMSPV_MASK_COMPLEMENT)
    assert S.spmspv_device_status(Ad.handle) == 0
    assert k == ref.idx.shape[0]
    compare(1, ref, yi.cpu().numpy(), yv.cpu().numpy())
    assert S.spmspv_last_work(Ad.handle) == ref.nmult
    Ad.close()
