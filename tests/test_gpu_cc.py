"""Connected components on the GPU (label propagation over SpMSpV rounds)
against the reference: labels bit for bit on R-MAT, a fragmented random graph
and a grid with removed edges, under every push schedule."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import need_gpu
from test_oracle_cc import sym_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = need_gpu()
    from paper_1610_07902_gb300 import spmspv as S
    S.load()
    return torch, S


def _graphs():
    yield "rmat13", synth.rmat(13, seed=6, values=False)
    colptr, rowidx = sym_graph(30000, 20000, 7, blocks=40)
    from types import SimpleNamespace
    yield "fragments", SimpleNamespace(m=30000, n=30000, colptr=colptr, rowidx=rowidx, val=None,
                                       nnz=rowidx.shape[0])
    yield "grid", synth.grid3d(24, 20, 16, 0.4, seed=5, values=False)


@pytest.mark.parametrize("sched", [None, 0, 2, 3, 5])
def test_cc_matches_reference(lib, sched):
    torch, S = lib
    for name, A in _graphs():
        Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
        labels = torch.empty(A.n, dtype=torch.int32, device="cuda")
        rounds = torch.zeros(1, dtype=torch.int32, device="cuda")
        opts = 0 if sched is None else S.SPMSPV_SCHED_OPT(sched)
        S.spmspv_cc(Ad.handle, labels, rounds, opts)
        ref, k = oracle.cc(A.colptr, A.rowidx)
        np.testing.assert_array_equal(labels.cpu().numpy(), ref, err_msg=name)
        assert 1 <= int(rounds.item()) <= A.n
        assert S.spmspv_device_status(Ad.handle) == 0
        # a second call on the same handle (graph reused) gives the same labels
        labels.fill_(-5)
        S.spmspv_cc(Ad.handle, labels, None, opts)
        np.testing.assert_array_equal(labels.cpu().numpy(), ref, err_msg=name)
        Ad.close()


def test_cc_rejects_directed_handles(lib):
    torch, S = lib
    A = synth.rmat(8, seed=1)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val)  # no symmetry flag
    labels = torch.empty(A.n, dtype=torch.int32, device="cuda")
    with pytest.raises(S.SpmspvError):
        S.spmspv_cc(Ad.handle, labels)
    Ad.close()


def test_cc_headline_graph(lib):
    """The headline R-MAT s22 graph, bit for bit against the reference."""
    torch, S = lib
    A = synth.rmat(22, seed=1, values=False)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
    labels = torch.empty(A.n, dtype=torch.int32, device="cuda")
    S.spmspv_cc(Ad.handle, labels)
    ref, k = oracle.cc(A.colptr, A.rowidx)
    np.testing.assert_array_equal(labels.cpu().numpy(), ref)
    assert S.spmspv_device_status(Ad.handle) == 0
    Ad.close()
