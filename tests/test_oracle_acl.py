"""Pins for the FP64 Andersen-Chung-Lang reference (oracle/acl.py).

The push is fixed by three facts that do not depend on how it is coded:
every push conserves mass (sum p + sum r = 1), every push keeps
p + pr(alpha, r) = pr(alpha, e_seed) for the lazy personalised PageRank
(a dense linear solve of its definition), and at termination every vertex
holds r(u) < eps d(u).  A hand-computed first step on a path pins the
constants (the 1/2 of the lazy walk, alpha on p, 1/d on the neighbours).
"""
import numpy as np
import pytest

from oracle import acl as oacl
import synth


def _sym_graph(n, avg, seed):
    rng = np.random.default_rng(seed)
    e = rng.integers(0, n, size=(n * avg // 2, 2))
    e = e[e[:, 0] != e[:, 1]]
    e = np.concatenate([e, e[:, ::-1]])
    key = np.unique(e[:, 1] * n + e[:, 0])
    col, row = key // n, key % n
    colptr = np.zeros(n + 1, np.int64)
    np.add.at(colptr, col + 1, 1)
    return np.cumsum(colptr), row


def test_first_step_on_a_path():
    # path 0 - 1 - 2, seed 1 (degree 2); alpha = 0.2
    colptr = np.array([0, 1, 3, 4])
    rowidx = np.array([1, 0, 2, 1])
    p, r, steps = oacl.acl(colptr, rowidx, 1, 0.2, 0.1, 1)
    assert steps == 1
    np.testing.assert_allclose(p, [0.0, 0.2, 0.0], atol=0)
    np.testing.assert_allclose(r, [0.2, 0.4, 0.2], rtol=1e-15)


def test_threshold_stops_at_once():
    colptr = np.array([0, 1, 3, 4])
    rowidx = np.array([1, 0, 2, 1])
    p, r, steps = oacl.acl(colptr, rowidx, 1, 0.2, 0.45, 50)  # 1 >= 0.45 * 2: one push
    assert steps == 1
    # after it: r(0) = 0.2 < 0.45, r(1) = 0.4 < 0.9, r(2) = 0.2 < 0.45
    p2, r2, steps2 = oacl.acl(colptr, rowidx, 1, 0.2, 0.51, 50)  # 1 < 0.51*2 -> nothing pushes
    assert steps2 == 0 and p2.sum() == 0 and r2[1] == 1.0


@pytest.mark.parametrize("seed", [0, 7, 123])
def test_invariants(seed):
    colptr, rowidx = _sym_graph(300, 6, seed)
    s = int(np.argmax(np.diff(colptr)))
    alpha, eps = 0.15, 1e-4
    target = oacl.lazy_pagerank(colptr, rowidx, alpha, np.eye(300)[s])
    for steps in (1, 2, 5, 1000):
        p, r, k = oacl.acl(colptr, rowidx, s, alpha, eps, steps)
        assert abs(p.sum() + r.sum() - 1.0) < 1e-12
        assert (p >= 0).all() and (r >= 0).all()
        rhs = p + oacl.lazy_pagerank(colptr, rowidx, alpha, r)
        np.testing.assert_allclose(rhs, target, atol=1e-12)
    deg = np.diff(colptr)
    assert k < 1000
    assert ((r < eps * deg) | (deg == 0)).all()
    # the approximation error is bounded by the residual: |p - pr|_1 <= sum r
    assert np.abs(p - target).sum() <= r.sum() + 1e-12


def test_isolated_seed_never_pushes():
    colptr = np.array([0, 0, 1, 2])
    rowidx = np.array([2, 1])
    p, r, k = oacl.acl(colptr, rowidx, 0, 0.15, 1e-6, 10)
    assert k == 0 and r[0] == 1.0 and p.sum() == 0


ACL_MUTANTS = {
    "not_lazy": ("r[u] = (1.0 - alpha) * r[u] / 2.0", "r[u] = 0.0"),
    "no_half_on_x": ("x[u] = (1.0 - alpha) * r[u] / (2.0 * deg[u])", "x[u] = (1.0 - alpha) * r[u] / deg[u]"),
    "alpha_swapped": ("p[u] += alpha * r[u]", "p[u] += (1.0 - alpha) * r[u]"),
    "strict_threshold": ("r[u] >= eps * deg[u]", "r[u] > eps * deg[u]"),
    "sequential_push": ("        for u, xu in x.items():\n            for q in range(colptr[u], colptr[u + 1]):\n                r[rowidx[q]] += xu\n",
                        "            for q in range(colptr[u], colptr[u + 1]):\n                r[rowidx[q]] += x[u]\n"),
}


def _pins_fail(mod):
    checks = []
    colptr = np.array([0, 1, 3, 4])
    rowidx = np.array([1, 0, 2, 1])
    p, r, k = mod.acl(colptr, rowidx, 1, 0.2, 0.1, 1)
    checks.append(np.allclose(p, [0, 0.2, 0]) and np.allclose(r, [0.2, 0.4, 0.2]))
    p, r, k = mod.acl(colptr, rowidx, 1, 0.2, 0.5, 50)  # r = 1 sits exactly on eps * d
    checks.append(k == 1)
    colptr, rowidx = _sym_graph(120, 6, 3)
    s = int(np.argmax(np.diff(colptr)))
    target = oacl.lazy_pagerank(colptr, rowidx, 0.15, np.eye(120)[s])
    p, r, k = mod.acl(colptr, rowidx, s, 0.15, 1e-4, 3)
    checks.append(abs(p.sum() + r.sum() - 1) < 1e-12)
    checks.append(np.allclose(p + oacl.lazy_pagerank(colptr, rowidx, 0.15, r), target, atol=1e-12))
    # synchronous: the seed's neighbours push from the residual the step started with
    colptr = np.array([0, 2, 4, 6])  # triangle
    rowidx = np.array([1, 2, 0, 2, 0, 1])
    p, r, k = mod.acl(colptr, rowidx, 0, 0.2, 0.05, 2)
    checks.append(np.allclose(p, [0.2 + 0.2 * 0.4, 0.2 * 0.2, 0.2 * 0.2]))
    return not all(checks)


def test_the_pins_catch_planted_slips():
    import inspect
    import types
    src = inspect.getsource(oacl)
    assert not _pins_fail(oacl)
    for name, (old, new) in ACL_MUTANTS.items():
        assert src.count(old) == 1, name
        mod = types.ModuleType("acl_" + name)
        exec(compile(src.replace(old, new), name, "exec"), mod.__dict__)
        assert _pins_fail(mod), name


@pytest.mark.parametrize("seed", [0, 7, 123])
def test_trace_form_equals_the_loop_form(seed):
    """acl_trace (whole-array steps, for large graphs) against acl(), whose
    arithmetic the pins above fix: the same p, r and step count to FP64
    rounding, and p(v) > 0 exactly where v pushed."""
    colptr, rowidx = _sym_graph(300, 6, seed)
    for s in (int(np.argmax(np.diff(colptr))), 5):
        for eps, steps in ((1e-4, 1000), (1e-3, 3), (1e-6, 1000)):
            p, r, k = oacl.acl(colptr, rowidx, s, 0.15, eps, steps)
            p2, r2, k2, pushes, margin = oacl.acl_trace(colptr, rowidx, s, 0.15, eps, steps)
            assert k2 == k
            np.testing.assert_allclose(p2, p, rtol=1e-12, atol=1e-15)
            np.testing.assert_allclose(r2, r, rtol=1e-12, atol=1e-15)
            assert ((p2 > 0) == (pushes > 0)).all()
            assert (pushes <= k).all() and (margin >= 0).all()


def test_trace_margins_by_hand():
    # path 0 - 1 - 2, seed 1, eps = 0.45 (thresholds 0.45, 0.9, 0.45): one
    # push at step 0 (margin |1 - 0.9| / 0.9), then r = (0.2, 0.4, 0.2)
    # leaves every vertex 5/9 below its threshold and nothing pushes
    colptr = np.array([0, 1, 3, 4])
    rowidx = np.array([1, 0, 2, 1])
    p, r, k, pushes, margin = oacl.acl_trace(colptr, rowidx, 1, 0.2, 0.45, 50)
    assert k == 1
    np.testing.assert_array_equal(pushes, [0, 1, 0])
    np.testing.assert_allclose(margin, [5 / 9, 1 / 9, 5 / 9], rtol=1e-12)
