"""Pins for the connected-components reference (oracle_cc in oracle/oracle.c).

label[v] must be the smallest vertex id of v's component: checked against
scipy's connected components (relabelled to component minima), against a
hand-made graph, and against the invariants that hold for any correct answer
(label[v] <= v, labels are fixed points, every edge joins equal labels).
"""
import numpy as np
import pytest

import oracle


def sym_graph(n, m_edges, seed, blocks=1):
    """Random undirected graph made of `blocks` disjoint vertex ranges."""
    rng = np.random.default_rng(seed)
    edges = []
    size = n // blocks
    for b in range(blocks):
        lo = b * size
        hi = n if b == blocks - 1 else lo + size
        e = rng.integers(lo, hi, size=(m_edges // blocks, 2))
        edges.append(e[e[:, 0] != e[:, 1]])
    e = np.concatenate(edges)
    e = np.concatenate([e, e[:, ::-1]])
    key = np.unique(e[:, 1].astype(np.int64) * n + e[:, 0])
    col, row = key // n, key % n
    colptr = np.zeros(n + 1, np.int64)
    np.add.at(colptr, col + 1, 1)
    return np.cumsum(colptr).astype(np.int32), row.astype(np.int32)


def min_labels_scipy(colptr, rowidx):
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    n = colptr.shape[0] - 1
    G = sp.csc_matrix((np.ones(rowidx.shape[0]), rowidx, colptr), shape=(n, n))
    k, comp = connected_components(G, directed=False)
    first = np.full(k, n, np.int64)
    np.minimum.at(first, comp, np.arange(n))
    return first[comp].astype(np.int32), k


def test_hand_graph():
    # components {0,2,5}, {1,4}, {3}, {6,7,8}: edges 0-5, 5-2, 4-1, 6-8, 8-7
    n = 9
    pairs = [(0, 5), (5, 2), (4, 1), (6, 8), (8, 7)]
    cols = [[] for _ in range(n)]
    for a, b in pairs:
        cols[a].append(b)
        cols[b].append(a)
    colptr = np.concatenate([[0], np.cumsum([len(c) for c in cols])]).astype(np.int32)
    rowidx = np.concatenate([sorted(c) for c in cols if c]).astype(np.int32)
    label, k = oracle.cc(colptr, rowidx)
    np.testing.assert_array_equal(label, [0, 1, 0, 3, 1, 0, 6, 6, 6])
    assert k == 4


@pytest.mark.parametrize("n,edges,blocks,seed", [(300, 200, 1, 1), (2000, 3000, 5, 2),
                                                 (5000, 2500, 1, 3), (1000, 8000, 10, 4)])
def test_against_scipy_and_invariants(n, edges, blocks, seed):
    colptr, rowidx = sym_graph(n, edges, seed, blocks)
    label, k = oracle.cc(colptr, rowidx)
    ref, kref = min_labels_scipy(colptr, rowidx)
    np.testing.assert_array_equal(label, ref)
    assert k == kref
    v = np.arange(n)
    assert (label <= v).all() and (label[label] == label).all()
    col_of = np.repeat(v, np.diff(colptr))
    assert (label[rowidx] == label[col_of]).all()


def test_edgeless_graph():
    label, k = oracle.cc(np.zeros(6, np.int32), np.zeros(0, np.int32))
    np.testing.assert_array_equal(label, np.arange(5))
    assert k == 5
