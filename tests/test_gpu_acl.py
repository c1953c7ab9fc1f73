"""Andersen-Chung-Lang push (batched lanes and the persistent form) against the
FP64 reference.

The pushing sets are decided in FP32 on the device and in FP64 in the
reference, so a vertex whose residual sits within rounding of eps*d(u) can
push on one side only.  What must hold regardless is checked tightly: mass
conservation, non-negativity and the termination rule.  The vectors are
compared element by element (gpu_util.acl_compare): every vertex within a
relative 1e-4 of the FP64 value when no decision came near its threshold,
and otherwise every vertex beyond two hops of the near ones.
"""
import numpy as np
import pytest

import synth
from gpu_util import acl_compare, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = need_gpu()
    from paper_1610_07902_gb300 import spmspv as S
    S.load()
    return torch, S


@pytest.mark.parametrize("graph,lanes", [("rmat", 4), ("grid", 1), ("grid", 8), ("rmat", -1), ("grid", -1)])
def test_acl_matches_reference(lib, graph, lanes):
    # lanes -1: the persistent form (SPMSPV_LANES_PERSISTENT)
    torch, S = lib
    assert S.SPMSPV_LANES_PERSISTENT == -1
    A = synth.rmat(11, seed=5, values=False) if graph == "rmat" else synth.grid3d(12, 12, 8, 0.2, values=False)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None, flags=S.SPMSPV_CSC_SYMMETRIC)
    seeds = synth.sources(A.colptr, 12, seed=6).astype(np.int32)
    B = seeds.shape[0]
    alpha, eps = 0.15, 1e-5
    p = torch.empty(B * A.n, dtype=torch.float32, device="cuda")
    r = torch.empty(B * A.n, dtype=torch.float32, device="cuda")
    k = torch.zeros(1, dtype=torch.int32, device="cuda")
    S.spmspv_acl(Ad.handle, B, torch.from_numpy(seeds).cuda(), alpha, eps, 10000, p, r, k, lanes)
    P = p.cpu().numpy().reshape(B, A.n).astype(np.float64)
    R = r.cpu().numpy().reshape(B, A.n).astype(np.float64)
    deg = np.diff(A.colptr).astype(np.float64)
    assert 0 < int(k.item()) < 10000
    for b in range(B):
        assert abs(P[b].sum() + R[b].sum() - 1.0) < 1e-5, b
        assert (P[b] >= 0).all() and (R[b] >= 0).all()
        assert ((R[b] < eps * deg * (1 + 1e-4)) | ((deg == 0) & (R[b] == 0))).all(), b
        acl_compare(P[b], R[b], A.colptr, A.rowidx, int(seeds[b]), alpha, eps, 10000)
    assert S.spmspv_device_status(Ad.handle) == 0
    Ad.close()


def test_acl_rejects_weighted_and_bad_args(lib):
    torch, S = lib
    A = synth.rmat(8, seed=2)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val, flags=S.SPMSPV_CSC_SYMMETRIC)
    p = torch.empty(A.n, dtype=torch.float32, device="cuda")
    seeds = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(S.SpmspvError):
        S.spmspv_acl(Ad.handle, 1, seeds, 0.15, 1e-6, 10, p, p.clone(), None, 2)
    Ad.close()
    Au = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None, flags=S.SPMSPV_CSC_SYMMETRIC)
    for alpha, eps in ((0.0, 1e-6), (1.0, 1e-6), (0.15, 0.0)):
        with pytest.raises(S.SpmspvError):
            S.spmspv_acl(Au.handle, 1, seeds, alpha, eps, 10, p, p.clone(), None, 2)
    Au.close()
