"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test ties oracle/oracle.c to something independent of it: the dense
matrix-vector closed form (numpy), brute force over every input subset,
special vectors with known answers, scipy.sparse, the multiply-count
invariant of Sec. II-D, a textbook queue BFS, scipy's shortest paths and
the Manhattan-distance closed form of an intact grid.  A plausible slip in
the oracle (a dropped product, a flipped min, a wrong mask polarity, a
transposed operand) fails at least one of them; test_oracle_mutants.py
checks that claim by planting such slips in copies of the oracle.
"""
from collections import deque
from fractions import Fraction
import zlib

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import oracle
import synth

INT_MAX = np.iinfo(np.int32).max


def random_csc(rng, m, n, density, with_val=True, sorted_rows=True):
    """A random m-by-n CSC built from a dense pattern (numpy only)."""
    pat = rng.random((m, n)) < density
    colptr = np.zeros(n + 1, dtype=np.int32)
    rows = []
    for j in range(n):
        r = np.flatnonzero(pat[:, j]).astype(np.int32)
        if not sorted_rows:
            r = rng.permutation(r).astype(np.int32)
        rows.append(r)
        colptr[j + 1] = colptr[j] + r.shape[0]
    rowidx = np.concatenate(rows) if rows else np.zeros(0, np.int32)
    val = None
    if with_val:
        val = (rng.random(rowidx.shape[0]) * 2 - 1).astype(np.float32)
    return colptr, rowidx.astype(np.int32), val


def to_dense(m, colptr, rowidx, val):
    n = colptr.shape[0] - 1
    P = np.zeros((m, n), dtype=bool)
    D = np.zeros((m, n), dtype=np.float64)
    for j in range(n):
        for p in range(colptr[j], colptr[j + 1]):
            P[rowidx[p], j] = True
            D[rowidx[p], j] = 1.0 if val is None else float(val[p])
    return P, D


def dense_reference(semiring, P, D, x_idx, x_val, mask, complement):
    """y from the dense definition y(i) = (+)_j A(i,j) (x) x(j)."""
    m, n = P.shape
    xind = np.zeros(n, dtype=bool)
    xind[x_idx] = True
    present = (P.astype(np.int64) @ xind.astype(np.int64)) > 0
    if mask is not None:
        keep = (mask == 0) if complement else (mask != 0)
        present &= keep
    idx = np.flatnonzero(present).astype(np.int32)
    if semiring == oracle.PLUS_TIMES:
        xd = np.zeros(n, dtype=np.float64)
        xd[x_idx] = x_val.astype(np.float64)
        y = D @ xd
        ab = np.abs(D) @ np.abs(xd)
        return idx, y[idx], ab[idx]
    if semiring == oracle.MIN_SELECT2ND:
        xv = np.full(n, INT_MAX, dtype=np.int64)
        xv[x_idx] = x_val
        cand = np.where(P & xind[None, :], xv[None, :], INT_MAX)
        return idx, cand.min(axis=1)[idx].astype(np.int32), None
    return idx, None, None


SEMIRINGS = [oracle.PLUS_TIMES, oracle.MIN_SELECT2ND, oracle.OR_AND]


@pytest.mark.parametrize("semiring", SEMIRINGS)
@pytest.mark.parametrize("shape", [(1, 1), (7, 5), (5, 9), (33, 64), (64, 17)])
@pytest.mark.parametrize("density", [0.05, 0.3, 0.9])
@pytest.mark.parametrize("mask_mode", ["none", "complement", "structural"])
def test_dense_closed_form(semiring, shape, density, mask_mode):
    rng = np.random.default_rng(zlib.crc32(repr((semiring, shape, density, mask_mode)).encode()))
    m, n = shape
    colptr, rowidx, val = random_csc(rng, m, n, density, sorted_rows=False)
    P, D = to_dense(m, colptr, rowidx, val)
    for _ in range(4):
        f = int(rng.integers(0, n + 1))
        x_idx = rng.permutation(n)[:f].astype(np.int32)
        if semiring == oracle.PLUS_TIMES:
            x_val = (rng.random(f) * 2 - 1).astype(np.float32)
        else:
            x_val = rng.integers(-1000, 1000, size=f).astype(np.int32)
        mask = None if mask_mode == "none" else (rng.random(m) < 0.4).astype(np.uint8)
        comp = mask_mode == "complement"
        r = oracle.spmspv(m, colptr, rowidx, val, semiring, x_idx, x_val, mask, comp)
        ei, ev, eab = dense_reference(semiring, P, D, x_idx, x_val, mask, comp)
        np.testing.assert_array_equal(r.idx, ei)
        if semiring == oracle.PLUS_TIMES:
            np.testing.assert_allclose(r.val, ev, rtol=0, atol=1e-12 * max(1.0, eab.max(initial=0)))
            np.testing.assert_allclose(r.absum, eab, rtol=1e-12)
        elif semiring == oracle.MIN_SELECT2ND:
            np.testing.assert_array_equal(r.val, ev)


def test_bruteforce_all_subsets():
    """Every subset of the columns of an 6x8 matrix, checked by a pure-Python
    double loop over (i, j) pairs."""
    rng = np.random.default_rng(11)
    m, n = 6, 8
    colptr, rowidx, val = random_csc(rng, m, n, 0.45)
    entries = {}
    for j in range(n):
        for p in range(colptr[j], colptr[j + 1]):
            entries[(int(rowidx[p]), j)] = float(val[p])
    xvals = (rng.random(n) * 4 - 2).astype(np.float32)
    ivals = rng.integers(0, 50, size=n).astype(np.int32)
    for bits in range(1 << n):
        S = [j for j in range(n) if bits >> j & 1]
        x_idx = np.array(S, dtype=np.int32)
        exp_f, exp_i = {}, {}
        for i in range(m):
            for j in S:
                if (i, j) in entries:
                    exp_f[i] = exp_f.get(i, 0.0) + entries[(i, j)] * float(xvals[j])
                    exp_i[i] = min(exp_i.get(i, INT_MAX), int(ivals[j]))
        r = oracle.spmspv(m, colptr, rowidx, val, oracle.PLUS_TIMES, x_idx, xvals[x_idx])
        assert list(r.idx) == sorted(exp_f)
        np.testing.assert_allclose(r.val, [exp_f[i] for i in sorted(exp_f)], atol=1e-12)
        r = oracle.spmspv(m, colptr, rowidx, val, oracle.MIN_SELECT2ND, x_idx, ivals[x_idx])
        assert list(r.idx) == sorted(exp_i)
        assert list(r.val) == [exp_i[i] for i in sorted(exp_i)]
        r = oracle.spmspv(m, colptr, rowidx, val, oracle.OR_AND, x_idx)
        assert list(r.idx) == sorted(exp_i)


def test_exact_rational_sum_within_fp64_bound():
    """The FP64 accumulation is within (k-1) u64 sum|a x| of the exact
    rational sum (k = products into the row, u64 = 2^-53)."""
    rng = np.random.default_rng(5)
    m, n = 40, 60
    colptr, rowidx, val = random_csc(rng, m, n, 0.5)
    x_idx = rng.permutation(n)[:45].astype(np.int32)
    x_val = (rng.random(45) * 2 - 1).astype(np.float32)
    r = oracle.spmspv(m, colptr, rowidx, val, oracle.PLUS_TIMES, x_idx, x_val)
    exact, cnt = {}, {}
    for k, j in enumerate(x_idx):
        for p in range(colptr[j], colptr[j + 1]):
            i = int(rowidx[p])
            exact[i] = exact.get(i, Fraction(0)) + Fraction(float(val[p])) * Fraction(float(x_val[k]))
            cnt[i] = cnt.get(i, 0) + 1
    assert list(r.idx) == sorted(exact)
    for q, i in enumerate(r.idx):
        err = abs(Fraction(float(r.val[q])) - exact[int(i)])
        assert err <= Fraction(max(cnt[int(i)] - 1, 0)) * Fraction(2) ** -53 * Fraction(float(r.absum[q])) * 2


def test_multiply_count_invariant():
    """nmult = sum over x's indices of the column lengths (Sec. II-D), masks included."""
    A = synth.rmat(12, seed=3)
    deg = A.degrees()
    rng = np.random.default_rng(2)
    for f in [0, 1, 17, 500, A.n]:
        x_idx, x_val = synth.frontier(A.n, f, seed=f + 1)
        mask = (rng.random(A.m) < 0.5).astype(np.uint8)
        for semiring in SEMIRINGS:
            xv = x_val if semiring == oracle.PLUS_TIMES else x_idx
            r = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, semiring, x_idx, xv, mask, True)
            assert r.nmult == int(deg[x_idx].sum())


def test_unit_vector_gives_column():
    A = synth.erdos_renyi(2000, d=9, seed=4)
    for j in [0, 7, 1234, 1999]:
        r = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, oracle.PLUS_TIMES,
                          np.array([j], np.int32), np.array([2.5], np.float32))
        rows = A.rowidx[A.colptr[j]:A.colptr[j + 1]]
        vals = A.val[A.colptr[j]:A.colptr[j + 1]].astype(np.float64) * 2.5
        order = np.argsort(rows)
        np.testing.assert_array_equal(r.idx, rows[order])
        np.testing.assert_array_equal(r.val, vals[order])


def test_all_ones_gives_row_sums():
    """x = all ones: y(i) is the i-th row sum, computed here by a loop over
    the stored entries grouped by row."""
    A = synth.erdos_renyi(3000, d=5, m=2000, seed=6)
    x_idx = np.arange(A.n, dtype=np.int32)
    r = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, oracle.PLUS_TIMES, x_idx,
                      np.ones(A.n, np.float32))
    order = np.argsort(A.rowidx, kind="stable")
    rows_sorted = A.rowidx[order]
    vals_sorted = A.val[order].astype(np.float64)
    uniq, start = np.unique(rows_sorted, return_index=True)
    sums = np.array([vals_sorted[s:e].sum() for s, e in zip(start, list(start[1:]) + [len(order)])])
    np.testing.assert_array_equal(r.idx, uniq)
    np.testing.assert_allclose(r.val, sums, rtol=1e-12)


@pytest.mark.parametrize("with_mask", [False, True])
def test_against_scipy(with_mask):
    A = synth.rmat(13, seed=9)
    S = sp.csc_matrix((A.val.astype(np.float64), A.rowidx, A.colptr), shape=(A.m, A.n))
    Pat = sp.csc_matrix((np.ones(A.nnz, np.int64), A.rowidx, A.colptr), shape=(A.m, A.n))
    rng = np.random.default_rng(3)
    for f in [1, 100, 3000]:
        x_idx, x_val = synth.frontier(A.n, f, seed=f)
        xd = np.zeros(A.n)
        xd[x_idx] = x_val
        xi = np.zeros(A.n, np.int64)
        xi[x_idx] = 1
        mask = (rng.random(A.m) < 0.3).astype(np.uint8) if with_mask else None
        r = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, oracle.PLUS_TIMES, x_idx, x_val, mask)
        present = (Pat @ xi) > 0
        if with_mask:
            present &= mask == 0
        idx = np.flatnonzero(present)
        np.testing.assert_array_equal(r.idx, idx)
        np.testing.assert_allclose(r.val, (S @ xd)[idx], rtol=1e-10, atol=1e-12)


def test_edge_cases():
    rng = np.random.default_rng(8)
    colptr, rowidx, val = random_csc(rng, 10, 12, 0.3)
    # empty x
    r = oracle.spmspv(10, colptr, rowidx, val, oracle.PLUS_TIMES, np.zeros(0, np.int32),
                      np.zeros(0, np.float32))
    assert r.idx.shape[0] == 0 and r.nmult == 0
    # everything masked out
    x = np.arange(12, dtype=np.int32)
    r = oracle.spmspv(10, colptr, rowidx, val, oracle.MIN_SELECT2ND, x, x,
                      np.ones(10, np.uint8), True)
    assert r.idx.shape[0] == 0 and r.nmult == int(colptr[-1])
    # empty columns only
    cp0 = np.zeros(13, np.int32)
    r = oracle.spmspv(10, cp0, np.zeros(0, np.int32), None, oracle.OR_AND, x)
    assert r.idx.shape[0] == 0
    # a single full column of a tall matrix, pattern values (a = 1)
    cp = np.array([0, 0, 1000, 1000], np.int32)
    ri = rng.permutation(1000).astype(np.int32)
    r = oracle.spmspv(1000, cp, ri, None, oracle.PLUS_TIMES, np.array([1, 2], np.int32),
                      np.array([3.0, 4.0], np.float32))
    np.testing.assert_array_equal(r.idx, np.arange(1000))
    np.testing.assert_array_equal(r.val, np.full(1000, 3.0))
    # structural zero: products that cancel keep the index
    cp = np.array([0, 1, 2], np.int32)
    r = oracle.spmspv(1, cp, np.array([0, 0], np.int32), np.array([1.0, 1.0], np.float32),
                      oracle.PLUS_TIMES, np.array([0, 1], np.int32),
                      np.array([2.0, -2.0], np.float32))
    assert list(r.idx) == [0] and r.val[0] == 0.0
    # INT32_MAX is an ordinary value for (min, select2nd)
    r = oracle.spmspv(1, cp, np.array([0, 0], np.int32), None, oracle.MIN_SELECT2ND,
                      np.array([0], np.int32), np.array([INT_MAX], np.int32))
    assert list(r.idx) == [0] and r.val[0] == INT_MAX
    # duplicate and out-of-range x indices are caller errors
    with pytest.raises(ValueError):
        oracle.spmspv(10, colptr, rowidx, val, oracle.OR_AND, np.array([3, 3], np.int32))
    with pytest.raises(ValueError):
        oracle.spmspv(10, colptr, rowidx, val, oracle.OR_AND, np.array([12], np.int32))


def queue_bfs(colptr, rowidx, src):
    """Textbook FIFO BFS: levels, and every vertex's set of minimum-level neighbours."""
    n = colptr.shape[0] - 1
    level = [-1] * n
    level[src] = 0
    q = deque([src])
    while q:
        v = q.popleft()
        for p in range(colptr[v], colptr[v + 1]):
            u = int(rowidx[p])
            if level[u] < 0:
                level[u] = level[v] + 1
                q.append(u)
    return np.array(level, dtype=np.int32)


def check_parents(colptr, rowidx, level, parent, src):
    """parent[v] is the smallest-id neighbour of v one level closer (A symmetric)."""
    n = colptr.shape[0] - 1
    assert parent[src] == src and level[src] == 0
    for v in range(n):
        if level[v] <= 0:
            if level[v] < 0:
                assert parent[v] == -1
            continue
        nb = rowidx[colptr[v]:colptr[v + 1]]
        cands = nb[level[nb] == level[v] - 1]
        assert cands.shape[0] > 0
        assert parent[v] == cands.min()


GRAPHS = [
    ("rmat10", lambda: synth.rmat(10, seed=4)),
    ("rmat12", lambda: synth.rmat(12, seed=5)),
    ("grid2d", lambda: synth.grid3d(40, 30, 1, 0.1, seed=3)),
    ("grid3d", lambda: synth.grid3d(12, 11, 10, 0.05, seed=3)),
]


@pytest.mark.parametrize("name,make", GRAPHS)
def test_bfs_against_queue_bfs_and_scipy(name, make):
    A = make()
    for src in synth.sources(A.colptr, 3, seed=1):
        level, parent, nl, tm, sizes = oracle.bfs(A.colptr, A.rowidx, src)
        np.testing.assert_array_equal(level, queue_bfs(A.colptr, A.rowidx, src))
        G = sp.csc_matrix((np.ones(A.nnz), A.rowidx, A.colptr), shape=(A.n, A.n))
        d = csg.shortest_path(G, method="D", unweighted=True, indices=int(src))
        exp = np.where(np.isinf(d), -1, d).astype(np.int32)
        np.testing.assert_array_equal(level, exp)
        check_parents(A.colptr, A.rowidx, level, parent, src)
        # every reached vertex is expanded exactly once
        assert tm == int(A.degrees()[level >= 0].sum())
        assert nl == level.max() + 1
        np.testing.assert_array_equal(sizes, np.bincount(level[level >= 0]))


@pytest.mark.parametrize("name,make", GRAPHS)
def test_bfs_pull_equals_push(name, make):
    A = make()
    for src in synth.sources(A.colptr, 2, seed=5):
        l1, p1, n1, _, _ = oracle.bfs(A.colptr, A.rowidx, src)
        l2, p2, n2 = oracle.bfs_pull(A.colptr, A.rowidx, src)
        np.testing.assert_array_equal(l1, l2)
        np.testing.assert_array_equal(p1, p2)
        assert n1 == n2


def test_intact_grid_levels_are_manhattan_distance():
    X, Y, Z = 9, 8, 7
    A = synth.grid3d(X, Y, Z, 0.0)
    c = (4, 4, 3)
    src = c[0] * Y * Z + c[1] * Z + c[2]
    level, parent, nl, _, _ = oracle.bfs(A.colptr, A.rowidx, src)
    v = np.arange(A.n)
    x, y, z = v // (Y * Z), (v // Z) % Y, v % Z
    np.testing.assert_array_equal(level, np.abs(x - c[0]) + np.abs(y - c[1]) + np.abs(z - c[2]))
    assert nl == 4 + 4 + 3 + 1


def test_hand_worked_example():
    """tests/golden/hand_example_3cols_4buckets.json, values worked by hand."""
    from golden_util import load_hand_example
    g = load_hand_example()
    args = (g["m"], g["colptr"], g["rowidx"], g["val"])
    xi = np.array(g["x_idx"], np.int32)
    r = oracle.spmspv(*args, oracle.PLUS_TIMES, xi, np.array(g["x_val_plus_times"], np.float32))
    assert list(r.idx) == g["expect_plus_times"]["idx"]
    assert list(r.val) == g["expect_plus_times"]["val"]
    assert r.nmult == g["multiply_count"]
    r = oracle.spmspv(*args, oracle.MIN_SELECT2ND, xi, np.array(g["x_val_min_select2nd"], np.int32))
    assert list(r.idx) == g["expect_min_select2nd"]["idx"]
    assert list(r.val) == g["expect_min_select2nd"]["val"]
    r = oracle.spmspv(*args, oracle.OR_AND, xi)
    assert list(r.idx) == g["expect_or_and"]["idx"]
    mask = np.zeros(g["m"], np.uint8)
    mask[g["mask_rows"]] = 1
    r = oracle.spmspv(*args, oracle.PLUS_TIMES, xi, np.array(g["x_val_plus_times"], np.float32),
                      mask, True)
    assert list(r.idx) == g["expect_plus_times_complement_mask"]["idx"]
    assert list(r.val) == g["expect_plus_times_complement_mask"]["val"]
    r = oracle.spmspv(*args, oracle.PLUS_TIMES, xi, np.array(g["x_val_plus_times"], np.float32),
                      mask, False)
    assert list(r.idx) == g["expect_plus_times_structural_mask"]["idx"]
    assert list(r.val) == g["expect_plus_times_structural_mask"]["val"]
    # bucket occupancy of the products, k = floor(i * nb / m) (Algorithm 1, Step 1)
    sizes = [0] * 4
    for j in g["x_idx"]:
        for p in range(g["colptr"][j], g["colptr"][j + 1]):
            sizes[int(g["rowidx"][p]) * 4 // g["m"]] += 1
    assert sizes == g["bucket_sizes_nb4"]
