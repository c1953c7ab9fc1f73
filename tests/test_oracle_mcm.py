"""Pins for the maximum-matching reference (oracle_mcm in oracle/oracle.c).

The cardinality of a maximum matching is unique; it is pinned by brute force
over every edge subset of tiny graphs, by Koenig's theorem (it equals the
smallest vertex cover, found by brute force over vertex subsets), by scipy's
Hopcroft-Karp routine on random rectangular graphs, and by hand graphs whose
answer follows from the definition (a graph where the first greedy choice has
to be undone, complete bipartite graphs, a permutation, stars, no edges).
The matching itself is checked for validity: mates agree on both sides and
every matched pair is an edge.
"""
import itertools

import numpy as np
import pytest

import oracle


def bip_csc(m, n, pairs):
    """CSC of the m-by-n biadjacency matrix with an entry at every (row, col) pair."""
    cols = [set() for _ in range(n)]
    for i, j in pairs:
        cols[j].add(i)
    colptr = np.concatenate([[0], np.cumsum([len(c) for c in cols])]).astype(np.int32)
    rowidx = np.array([r for c in cols for r in sorted(c)], dtype=np.int32)
    return colptr, rowidx


def random_bip(m, n, edges, seed):
    rng = np.random.default_rng(seed)
    return bip_csc(m, n, zip(rng.integers(0, m, edges).tolist(), rng.integers(0, n, edges).tolist()))


def check_valid(m, colptr, rowidx, mate_r, mate_c, size):
    n = colptr.shape[0] - 1
    assert mate_r.shape == (m,) and mate_c.shape == (n,)
    matched = 0
    for j in range(n):
        i = mate_c[j]
        if i >= 0:
            matched += 1
            assert mate_r[i] == j, "mates disagree"
            assert i in rowidx[colptr[j]:colptr[j + 1]], "matched pair is not an edge"
    assert ((mate_r >= 0).sum()) == matched == size


def brute_max_matching(m, colptr, rowidx):
    n = colptr.shape[0] - 1
    edges = [(int(rowidx[p]), j) for j in range(n) for p in range(colptr[j], colptr[j + 1])]
    best = 0
    for k in range(len(edges), 0, -1):
        if k <= best:
            break
        for sub in itertools.combinations(edges, k):
            rows = {e[0] for e in sub}
            cols = {e[1] for e in sub}
            if len(rows) == k and len(cols) == k:
                return k
    return best


def brute_min_vertex_cover(m, colptr, rowidx):
    n = colptr.shape[0] - 1
    edges = [(int(rowidx[p]), j) for j in range(n) for p in range(colptr[j], colptr[j + 1])]
    for k in range(m + n + 1):
        for cover in itertools.combinations(range(m + n), k):
            s = set(cover)
            if all(i in s or (m + j) in s for i, j in edges):
                return k
    return m + n


def test_first_greedy_choice_must_be_undone():
    # column 0 sees rows 0 and 1, column 1 only row 0: column 0 has to give row 0 up
    colptr, rowidx = bip_csc(2, 2, [(0, 0), (1, 0), (0, 1)])
    mate_r, mate_c, k = oracle.mcm(2, colptr, rowidx)
    assert k == 2
    np.testing.assert_array_equal(mate_c, [1, 0])
    np.testing.assert_array_equal(mate_r, [1, 0])


def test_long_alternating_path():
    # columns 0..n-2 see rows j and j+1 and take row j; the last column sees
    # only row 0, so its augmenting path runs through every other column
    n = 40
    pairs = [(j, j) for j in range(n - 1)] + [(j + 1, j) for j in range(n - 1)] + [(0, n - 1)]
    colptr, rowidx = bip_csc(n, n, pairs)
    mate_r, mate_c, k = oracle.mcm(n, colptr, rowidx)
    assert k == n
    check_valid(n, colptr, rowidx, mate_r, mate_c, k)
    np.testing.assert_array_equal(mate_c, list(range(1, n)) + [0])


@pytest.mark.parametrize("m,n", [(3, 5), (5, 3), (4, 4)])
def test_complete_bipartite(m, n):
    colptr, rowidx = bip_csc(m, n, [(i, j) for i in range(m) for j in range(n)])
    mate_r, mate_c, k = oracle.mcm(m, colptr, rowidx)
    assert k == min(m, n)
    check_valid(m, colptr, rowidx, mate_r, mate_c, k)


def test_permutation_stars_and_no_edges():
    perm = np.random.default_rng(1).permutation(50)
    colptr, rowidx = bip_csc(50, 50, [(int(perm[j]), j) for j in range(50)])
    mate_r, mate_c, k = oracle.mcm(50, colptr, rowidx)
    assert k == 50
    np.testing.assert_array_equal(mate_c, perm)
    assert oracle.mcm(9, *bip_csc(9, 1, [(i, 0) for i in range(9)]))[2] == 1
    assert oracle.mcm(1, *bip_csc(1, 9, [(0, j) for j in range(9)]))[2] == 1
    mate_r, mate_c, k = oracle.mcm(6, np.zeros(5, np.int32), np.zeros(0, np.int32))
    assert k == 0 and (mate_r == -1).all() and (mate_c == -1).all()


@pytest.mark.parametrize("seed", range(8))
def test_bruteforce_and_koenig_tiny(seed):
    rng = np.random.default_rng(seed)
    m, n = int(rng.integers(2, 6)), int(rng.integers(2, 6))
    colptr, rowidx = random_bip(m, n, int(rng.integers(3, 11)), seed)
    mate_r, mate_c, k = oracle.mcm(m, colptr, rowidx)
    check_valid(m, colptr, rowidx, mate_r, mate_c, k)
    assert k == brute_max_matching(m, colptr, rowidx)
    assert k == brute_min_vertex_cover(m, colptr, rowidx)


@pytest.mark.parametrize("m,n,edges,seed", [(300, 200, 500, 1), (1000, 1500, 2200, 2),
                                            (4000, 4000, 12000, 3), (2000, 3000, 30000, 4)])
def test_against_scipy_hopcroft_karp(m, n, edges, seed):
    import scipy.sparse as sp
    from scipy.sparse.csgraph import maximum_bipartite_matching
    colptr, rowidx = random_bip(m, n, edges, seed)
    mate_r, mate_c, k = oracle.mcm(m, colptr, rowidx)
    check_valid(m, colptr, rowidx, mate_r, mate_c, k)
    B = sp.csc_matrix((np.ones(rowidx.shape[0]), rowidx, colptr), shape=(m, n)).tocsr()
    ref = maximum_bipartite_matching(B, perm_type="column")
    assert k == int((ref >= 0).sum())
