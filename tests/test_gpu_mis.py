"""Maximal independent set on the GPU (Luby's rounds with fixed priorities,
two masked SpMSpVs per round) against the reference: membership bit for bit
on R-MAT, a fragmented random graph, a grid with removed edges, a complete
graph, an edgeless graph and a long path whose increasing priorities take one
round per two vertices, under every push schedule."""
from types import SimpleNamespace

import numpy as np
import pytest

import oracle
import synth
from gpu_util import need_gpu
from test_oracle_cc import sym_graph
from test_oracle_mis import csc_from_pairs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = need_gpu()
    from paper_1610_07902_gb300 import spmspv as S
    S.load()
    return torch, S


def _ns(colptr, rowidx):
    n = colptr.shape[0] - 1
    return SimpleNamespace(m=n, n=n, colptr=colptr, rowidx=rowidx, val=None, nnz=rowidx.shape[0])


def _graphs():
    yield "rmat13", synth.rmat(13, seed=6, values=False)
    yield "fragments", _ns(*sym_graph(30000, 20000, 7, blocks=40))
    yield "grid", synth.grid3d(24, 20, 16, 0.4, seed=5, values=False)
    yield "complete300", _ns(*csc_from_pairs(300, [(a, b) for a in range(300) for b in range(a)]))
    yield "edgeless", _ns(np.zeros(1001, np.int32), np.zeros(0, np.int32))


def _run(torch, S, A, prio, opts):
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
    d_prio = torch.from_numpy(prio).cuda()
    in_set = torch.full((A.n,), -3, dtype=torch.int32, device="cuda")
    rounds = torch.zeros(1, dtype=torch.int32, device="cuda")
    S.spmspv_mis(Ad.handle, d_prio, in_set, rounds, opts)
    got = in_set.cpu().numpy()
    r = int(rounds.item())
    assert S.spmspv_device_status(Ad.handle) == 0
    # a second call on the same handle (graph and buffers reused)
    in_set.fill_(7)
    S.spmspv_mis(Ad.handle, d_prio, in_set, None, opts)
    again = in_set.cpu().numpy()
    Ad.close()
    return got, again, r


@pytest.mark.parametrize("sched", [None, 0, 2, 3, 5])
def test_mis_matches_reference(lib, sched):
    torch, S = lib
    opts = 0 if sched is None else S.SPMSPV_SCHED_OPT(sched)
    for k, (name, A) in enumerate(_graphs()):
        prio = np.random.default_rng(50 + k).permutation(A.n).astype(np.int32)
        if k % 2:
            prio = prio * 5 - 2 * A.n  # negative and positive, gaps between values
        got, again, rounds = _run(torch, S, A, prio, opts)
        ref, size = oracle.mis(A.colptr, A.rowidx, prio)
        np.testing.assert_array_equal(got, ref, err_msg=name)
        np.testing.assert_array_equal(again, ref, err_msg=name)
        assert 1 <= rounds <= A.n
        if name == "complete300":
            assert size == 1
        if name == "edgeless":
            assert size == A.n and rounds == 1


def test_mis_long_path_takes_many_rounds(lib):
    torch, S = lib
    n = 3001
    A = _ns(*csc_from_pairs(n, [(v, v + 1) for v in range(n - 1)]))
    prio = np.arange(n, dtype=np.int32)
    got, _, rounds = _run(torch, S, A, prio, 0)
    ref, size = oracle.mis(A.colptr, A.rowidx, prio)
    np.testing.assert_array_equal(got, ref)
    assert size == (n + 1) // 2 and rounds == (n + 1) // 2


def test_mis_with_self_loops_and_hubs(lib):
    torch, S = lib
    # R-MAT s14 (hub columns from the skew) with a self loop on every third vertex
    R = synth.rmat(14, seed=9, values=False)
    col = np.repeat(np.arange(R.n), np.diff(R.colptr))
    A = _ns(*csc_from_pairs(R.n, list(zip(col.tolist(), R.rowidx.tolist())),
                            self_loops=range(0, R.n, 3)))
    assert (np.repeat(np.arange(A.n), np.diff(A.colptr)) == A.rowidx).sum() == (R.n + 2) // 3
    prio = np.random.default_rng(3).permutation(A.n).astype(np.int32)
    got, _, _ = _run(torch, S, A, prio, 0)
    ref, _ = oracle.mis(A.colptr, A.rowidx, prio)
    np.testing.assert_array_equal(got, ref)


def test_mis_rejects_bad_calls(lib):
    torch, S = lib
    A = synth.rmat(8, seed=1)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val)  # no symmetry flag
    prio = torch.arange(A.n, dtype=torch.int32, device="cuda")
    in_set = torch.empty(A.n, dtype=torch.int32, device="cuda")
    with pytest.raises(S.SpmspvError):
        S.spmspv_mis(Ad.handle, prio, in_set)
    Ad.close()
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
    with pytest.raises(S.SpmspvError):
        S.spmspv_mis(Ad.handle, prio, in_set, None, S.SPMSPV_SCHED_AUTO)
    with pytest.raises(S.SpmspvError):
        S.spmspv_mis(Ad.handle, None, in_set)
    with pytest.raises(S.SpmspvError):
        S.spmspv_mis(Ad.handle, prio, in_set, None, S.SPMSPV_SCHED_OPT(7))
    Ad.close()


def test_mis_headline_graph(lib):
    """The headline R-MAT s22 graph, bit for bit against the reference."""
    torch, S = lib
    A = synth.rmat(22, seed=1, values=False)
    prio = np.random.default_rng(22).permutation(A.n).astype(np.int32)
    got, _, rounds = _run(torch, S, A, prio, 0)
    ref, size = oracle.mis(A.colptr, A.rowidx, prio)
    np.testing.assert_array_equal(got, ref)
    assert rounds >= 1
