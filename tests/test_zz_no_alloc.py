"""The allocation-free entry point (spmspv_run_noalloc) against the handle path.

spmspv_run_noalloc serves callers that cannot call cudaMalloc: it keeps its
scratch in one library-owned device array instead of a handle's workspace.
This file is named so that pytest collects it last; the test passes both in
a fresh process and after every other test.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import FP_TOL, need_gpu

pytestmark = pytest.mark.gpu


def test_noalloc_matches_handle_path_on_two_calls():
    torch = need_gpu()
    from paper_1610_07902_gb300 import spmspv as S
    S.load()
    A = synth.erdos_renyi(60000, d=12, seed=21)          # nnz(A) ~ 720K <= 2^20
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val)
    cap = A.m
    for call, (f, semiring) in enumerate([(3000, S.SPMSPV_PLUS_TIMES_F32),
                                          (20000, S.SPMSPV_PLUS_TIMES_F32)]):
        x_idx, xf = synth.frontier(A.n, f, seed=100 + call)
        xi = torch.from_numpy(x_idx).cuda()
        xv = torch.from_numpy(xf).cuda()
        # the existing entry point (handle with its own workspace)
        yi_h, yv_h, k_h = Ad.multiply(semiring, xi, xv)
        # the allocation-free one
        yi = torch.empty(cap, dtype=torch.int32, device="cuda")
        yv = torch.empty(cap, dtype=torch.float32, device="cuda")
        nz = torch.zeros(1, dtype=torch.int32, device="cuda")
        S.spmspv_run_noalloc(A.m, A.n, A.nnz, Ad.colptr, Ad.rowidx, Ad.val, S.SPMSPV_VAL_F32,
                             semiring, xi, xv, f, None, 0, yi, yv, cap, nz)
        k = int(nz.item())
        assert k == k_h
        np.testing.assert_array_equal(yi[:k].cpu().numpy(), yi_h.cpu().numpy())
        # both within the parity tolerance of the FP64 oracle, so within 2x of each other
        ref = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, oracle.PLUS_TIMES, x_idx, xf)
        diff = np.abs(yv[:k].cpu().numpy().astype(np.float64) - yv_h.cpu().numpy())
        assert np.all(diff <= 2 * FP_TOL * ref.absum)
    Ad.close()


def test_noalloc_rejects_sizes_beyond_its_maximum():
    torch = need_gpu()
    from paper_1610_07902_gb300 import spmspv as S
    S.load()
    cp = torch.zeros(2, dtype=torch.int32, device="cuda")
    x = torch.zeros(1, dtype=torch.int32, device="cuda")
    y = torch.zeros(1, dtype=torch.int32, device="cuda")
    nz = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(S.SpmspvError) as e:
        S.spmspv_run_noalloc((1 << 22) + 1, 1, 0, cp, None, None, S.SPMSPV_VAL_NONE,
                             S.SPMSPV_OR_AND_BOOL, x, None, 1, None, 0, y, None, 1, nz)
    assert e.value.code == S.SPMSPV_ERR_UNSUPPORTED and "maximum" in str(e.value)
    with pytest.raises(S.SpmspvError) as e:
        S.spmspv_run_noalloc(4, 1, (1 << 20) + 1, cp, x, None, S.SPMSPV_VAL_NONE,
                             S.SPMSPV_OR_AND_BOOL, x, None, 1, None, 0, y, None, 1, nz)
    assert e.value.code == S.SPMSPV_ERR_UNSUPPORTED and "maximum" in str(e.value)
