"""Maximum bipartite matching on the GPU (phases of multi-source alternating
BFS over SpMSpV levels) against the reference.  Several maximum matchings can
exist, so the cardinality (unique) is compared with the reference and the
matching itself is checked for validity: both mate arrays agree and every
matched pair is an edge.  R-MAT (square), rectangular random graphs of both
orientations, a grid, a complete bipartite graph, a graph without edges and
a chain whose last column needs a long augmenting path, under every push
schedule."""
from types import SimpleNamespace

import numpy as np
import pytest

import oracle
import synth
from gpu_util import need_gpu
from test_oracle_mcm import bip_csc, random_bip

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = need_gpu()
    from paper_1610_07902_gb300 import spmspv as S
    S.load()
    return torch, S


def _ns(m, colptr, rowidx):
    return SimpleNamespace(m=m, n=colptr.shape[0] - 1, colptr=colptr, rowidx=rowidx, val=None,
                           nnz=rowidx.shape[0])


def _graphs():
    yield "rmat13", synth.rmat(13, seed=6, values=False)
    yield "tall", _ns(30000, *random_bip(30000, 20000, 45000, 8))
    yield "wide", _ns(12000, *random_bip(12000, 25000, 40000, 9))
    yield "grid", synth.grid3d(24, 20, 16, 0.3, seed=5, values=False)
    yield "complete50x80", _ns(50, *bip_csc(50, 80, [(i, j) for i in range(50) for j in range(80)]))
    yield "no_edges", _ns(700, np.zeros(501, np.int32), np.zeros(0, np.int32))
    n = 2000
    chain = [(j, j) for j in range(n - 1)] + [(j + 1, j) for j in range(n - 1)] + [(0, n - 1)]
    yield "chain", _ns(n, *bip_csc(n, n, chain))


def check_matching(A, mate_r, mate_c):
    matched = np.flatnonzero(mate_c >= 0)
    rows = mate_c[matched]
    assert (mate_r[rows] == matched).all(), "mates disagree"
    assert ((mate_r >= 0).sum()) == matched.shape[0]
    assert np.unique(rows).shape[0] == rows.shape[0]
    col = np.repeat(np.arange(A.n, dtype=np.int64), np.diff(A.colptr))
    edges = col * A.m + A.rowidx.astype(np.int64)
    assert np.isin(matched.astype(np.int64) * A.m + rows, edges).all(), "a matched pair is not an edge"
    return matched.shape[0]


def _run(torch, S, A, opts):
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None)
    mate_r = torch.full((A.m,), -7, dtype=torch.int32, device="cuda")
    mate_c = torch.full((A.n,), -7, dtype=torch.int32, device="cuda")
    card = torch.zeros(1, dtype=torch.int32, device="cuda")
    phases = torch.zeros(1, dtype=torch.int32, device="cuda")
    S.spmspv_mcm(Ad.handle, mate_r, mate_c, card, phases, opts)
    out = (mate_r.cpu().numpy(), mate_c.cpu().numpy(), int(card.item()), int(phases.item()))
    assert S.spmspv_device_status(Ad.handle) == 0
    # a second call on the same handle (graph and buffers reused)
    S.spmspv_mcm(Ad.handle, mate_r, mate_c, card, None, opts)
    again = (mate_r.cpu().numpy(), mate_c.cpu().numpy(), int(card.item()))
    Ad.close()
    return out, again


@pytest.mark.parametrize("sched", [None, 0, 2, 3, 5])
def test_mcm_matches_reference_cardinality(lib, sched):
    torch, S = lib
    opts = 0 if sched is None else S.SPMSPV_SCHED_OPT(sched)
    for name, A in _graphs():
        (mate_r, mate_c, card, phases), again = _run(torch, S, A, opts)
        _, _, ref = oracle.mcm(A.m, A.colptr, A.rowidx)
        assert check_matching(A, mate_r, mate_c) == card == ref, name
        assert check_matching(A, again[0], again[1]) == again[2] == ref, name
        assert 0 <= phases <= min(A.m, A.n), name
        if name == "complete50x80":
            assert card == 50
        if name == "no_edges":
            assert card == 0 and (mate_r == -1).all() and (mate_c == -1).all()


def test_mcm_rmat16(lib):
    torch, S = lib
    A = synth.rmat(16, seed=1, values=False)
    (mate_r, mate_c, card, phases), _ = _run(torch, S, A, 0)
    _, _, ref = oracle.mcm(A.m, A.colptr, A.rowidx)
    assert check_matching(A, mate_r, mate_c) == card == ref
    assert phases >= 1


def test_mcm_rejects_bad_calls(lib):
    torch, S = lib
    A = synth.rmat(8, seed=1)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None)
    mate_r = torch.empty(A.m, dtype=torch.int32, device="cuda")
    mate_c = torch.empty(A.n, dtype=torch.int32, device="cuda")
    with pytest.raises(S.SpmspvError):
        S.spmspv_mcm(Ad.handle, None, mate_c)
    with pytest.raises(S.SpmspvError):
        S.spmspv_mcm(Ad.handle, mate_r, mate_c, None, None, S.SPMSPV_SCHED_AUTO)
    with pytest.raises(S.SpmspvError):
        S.spmspv_mcm(Ad.handle, mate_r, mate_c, None, None, S.SPMSPV_SCHED_OPT(9))
    Ad.close()
