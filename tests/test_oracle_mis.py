"""Pins for the maximal-independent-set reference (oracle_mis in oracle/oracle.c).

The reference keeps vertices greedily in order of increasing priority.  It is
pinned by hand graphs whose answer follows from the definition (path, star,
complete graph, edgeless graph), by brute force over every vertex subset of
tiny graphs (the greedy set is the one independent set in which every vertex
left out has a neighbour inside with a smaller priority), by a pure-Python
simulation of Luby's synchronous rounds with the same fixed priorities (a
different algorithm that reaches the same set), and by the invariants of any
maximal independent set.
"""
import itertools

import numpy as np
import pytest

import oracle


def csc_from_pairs(n, pairs, self_loops=()):
    cols = [set() for _ in range(n)]
    for a, b in pairs:
        if a != b:
            cols[a].add(b)
            cols[b].add(a)
    for v in self_loops:
        cols[v].add(v)
    colptr = np.concatenate([[0], np.cumsum([len(c) for c in cols])]).astype(np.int32)
    rowidx = np.array([r for c in cols for r in sorted(c)], dtype=np.int32)
    return colptr, rowidx


def random_graph(n, m_edges, seed):
    rng = np.random.default_rng(seed)
    e = rng.integers(0, n, size=(m_edges, 2))
    return csc_from_pairs(n, [tuple(x) for x in e])


def neighbours(colptr, rowidx, v):
    return [int(u) for u in rowidx[colptr[v]:colptr[v + 1]] if u != v]


def luby_rounds(colptr, rowidx, prio):
    """Luby's rounds with fixed priorities: every undecided vertex whose
    priority is below those of all its undecided neighbours joins; the
    neighbours of the joiners leave; repeat until nobody is undecided."""
    n = colptr.shape[0] - 1
    state = [0] * n  # 0 undecided, 1 in, 2 out
    rounds = 0
    while any(s == 0 for s in state):
        rounds += 1
        join = [v for v in range(n) if state[v] == 0 and
                all(prio[u] > prio[v] for u in neighbours(colptr, rowidx, v) if state[u] == 0)]
        assert join, "no local minimum among the undecided vertices"
        for v in join:
            state[v] = 1
        for v in join:
            for u in neighbours(colptr, rowidx, v):
                if state[u] == 0:
                    state[u] = 2
    return np.array([1 if s == 1 else 0 for s in state], dtype=np.int32), rounds


def check_invariants(colptr, rowidx, prio, in_set):
    n = colptr.shape[0] - 1
    for v in range(n):
        nb = neighbours(colptr, rowidx, v)
        if in_set[v]:
            assert not any(in_set[u] for u in nb), "two adjacent members"
        else:
            assert any(in_set[u] and prio[u] < prio[v] for u in nb), \
                "vertex %d left out without a smaller-priority member neighbour" % v


def test_path():
    colptr, rowidx = csc_from_pairs(4, [(0, 1), (1, 2), (2, 3)])
    in_set, k = oracle.mis(colptr, rowidx, np.array([1, 0, 3, 2], np.int32))
    np.testing.assert_array_equal(in_set, [0, 1, 0, 1])
    assert k == 2
    in_set, k = oracle.mis(colptr, rowidx, np.array([0, 1, 2, 3], np.int32))
    np.testing.assert_array_equal(in_set, [1, 0, 1, 0])


def test_star():
    colptr, rowidx = csc_from_pairs(6, [(0, v) for v in range(1, 6)])
    in_set, k = oracle.mis(colptr, rowidx, np.array([-5, 1, 2, 3, 4, 5], np.int32))
    np.testing.assert_array_equal(in_set, [1, 0, 0, 0, 0, 0])
    in_set, k = oracle.mis(colptr, rowidx, np.array([9, 1, 2, 3, 4, 5], np.int32))
    np.testing.assert_array_equal(in_set, [0, 1, 1, 1, 1, 1])
    assert k == 5


def test_complete_graph_keeps_the_smallest_priority():
    n = 7
    colptr, rowidx = csc_from_pairs(n, list(itertools.combinations(range(n), 2)))
    prio = np.array([40, 12, 33, 7, 25, 90, 11], np.int32)
    in_set, k = oracle.mis(colptr, rowidx, prio)
    assert k == 1 and in_set[3] == 1


def test_edgeless_graph_keeps_everything():
    in_set, k = oracle.mis(np.zeros(6, np.int32), np.zeros(0, np.int32),
                           np.array([5, 4, 3, 2, 1], np.int32))
    np.testing.assert_array_equal(in_set, np.ones(5))
    assert k == 5


def test_self_loops_change_nothing():
    pairs = [(0, 1), (1, 2), (2, 3), (3, 0), (1, 3)]
    prio = np.array([3, 1, 0, 2], np.int32)
    a = oracle.mis(*csc_from_pairs(4, pairs), prio)[0]
    b = oracle.mis(*csc_from_pairs(4, pairs, self_loops=(0, 1, 2, 3)), prio)[0]
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_tiny(seed):
    rng = np.random.default_rng(seed)
    n = 9
    colptr, rowidx = random_graph(n, int(rng.integers(4, 18)), seed)
    prio = rng.permutation(n).astype(np.int32) * 3 - 7
    in_set, k = oracle.mis(colptr, rowidx, prio)
    found = []
    for bits in range(1 << n):
        s = [(bits >> v) & 1 for v in range(n)]
        try:
            check_invariants(colptr, rowidx, prio, s)
        except AssertionError:
            continue
        found.append(s)
    assert len(found) == 1
    np.testing.assert_array_equal(in_set, found[0])
    assert k == sum(found[0])


@pytest.mark.parametrize("n,edges,seed", [(50, 120, 1), (400, 1600, 2), (1500, 3000, 3),
                                          (2000, 16000, 4)])
def test_against_luby_rounds(n, edges, seed):
    colptr, rowidx = random_graph(n, edges, seed)
    prio = np.random.default_rng(seed + 100).permutation(n).astype(np.int32)
    in_set, k = oracle.mis(colptr, rowidx, prio)
    ref, rounds = luby_rounds(colptr, rowidx, prio)
    np.testing.assert_array_equal(in_set, ref)
    assert k == int(ref.sum())
    check_invariants(colptr, rowidx, prio, in_set)


def test_repeated_priority_is_rejected():
    colptr, rowidx = csc_from_pairs(3, [(0, 1)])
    with pytest.raises(ValueError):
        oracle.mis(colptr, rowidx, np.array([1, 2, 1], np.int32))
