"""FP64 reference of the Andersen-Chung-Lang push (test infrastructure only).

Sec. I lists local graph clustering (Andersen, Chung and Lang) as one of
the algorithms that make one SpMSpV per step; the paper gives no algorithm
of its own, so this follows the synchronous push: per step every vertex
whose residual is at least eps times its degree pushes at once, from the
residuals the step started with.  Written from the definition of the push
on the lazy walk W = (I + A D^-1) / 2:

    push(u):  p(u) += alpha r(u);  r(u) <- (1 - alpha) r(u) / 2;
              r(v) += (1 - alpha) r(u) / (2 d(u))  for every neighbour v of u.

The neighbour update of a whole step is the product A x with
x(u) = (1 - alpha) r(u) / (2 d(u)) on the pushing set, which is the SpMSpV.
Plain loops over the active set; meant for graphs of up to a few thousand
vertices.
"""
import numpy as np


def acl(colptr, rowidx, seed, alpha, eps, max_steps):
    """Return (p, r, steps) for one seed on the unweighted graph in CSC form."""
    colptr = np.asarray(colptr, np.int64)
    rowidx = np.asarray(rowidx, np.int64)
    n = len(colptr) - 1
    deg = np.diff(colptr).astype(np.float64)
    p = np.zeros(n)
    r = np.zeros(n)
    r[seed] = 1.0
    steps = 0
    while steps < max_steps:
        active = [u for u in range(n) if deg[u] > 0 and r[u] >= eps * deg[u]]
        if not active:
            break
        x = {}
        for u in active:
            x[u] = (1.0 - alpha) * r[u] / (2.0 * deg[u])
            p[u] += alpha * r[u]
            r[u] = (1.0 - alpha) * r[u] / 2.0
        for u, xu in x.items():
            for q in range(colptr[u], colptr[u + 1]):
                r[rowidx[q]] += xu
        steps += 1
    return p, r, steps


def lazy_pagerank(colptr, rowidx, alpha, v):
    """pr(alpha, v) = alpha (I - (1 - alpha) W)^-1 v with W = (I + A D^-1) / 2.

    A dense solve of the personalised PageRank definition, independent of
    the push; ACL keeps p + pr(alpha, r) = pr(alpha, e_seed) after every push.
    """
    colptr = np.asarray(colptr, np.int64)
    n = len(colptr) - 1
    A = np.zeros((n, n))
    for j in range(n):
        for q in range(colptr[j], colptr[j + 1]):
            A[rowidx[q], j] += 1.0
    deg = np.diff(colptr).astype(np.float64)
    dinv = np.where(deg > 0, 1.0 / np.maximum(deg, 1.0), 0.0)
    W = 0.5 * (np.eye(n) + A * dinv[None, :])
    return alpha * np.linalg.solve(np.eye(n) - (1.0 - alpha) * W, np.asarray(v, np.float64))


def acl_trace(colptr, rowidx, seed, alpha, eps, max_steps):
    """The same synchronous push as acl(), with whole-array numpy steps, for
    graphs of millions of vertices; also returns, per vertex, how many steps
    it pushed in and how close its residual came to the push threshold.

    Returns (p, r, steps, pushes, margin): pushes int32[n]; margin[v] = the
    smallest |r(v) - eps d(v)| / (eps d(v)) over the steps at whose start v
    had a positive residual (inf if it never had one).  A vertex with a small
    margin is one whose push decision a lower-precision run may take the
    other way.  The neighbour update adds each step's contributions into r
    as one sum per vertex (r += A x), so p and r agree with acl() to FP64
    rounding, not bit for bit.
    """
    colptr = np.asarray(colptr, np.int64)
    rowidx = np.asarray(rowidx, np.int64)
    n = len(colptr) - 1
    deg = np.diff(colptr).astype(np.float64)
    thr = eps * deg
    p = np.zeros(n)
    r = np.zeros(n)
    r[seed] = 1.0
    pushes = np.zeros(n, np.int32)
    margin = np.full(n, np.inf)
    steps = 0
    while steps < max_steps:
        cand = np.flatnonzero((r > 0) & (deg > 0))
        margin[cand] = np.minimum(margin[cand], np.abs(r[cand] - thr[cand]) / thr[cand])
        active = cand[r[cand] >= thr[cand]]
        if active.size == 0:
            break
        ru = r[active]
        xu = (1.0 - alpha) * ru / (2.0 * deg[active])
        p[active] += alpha * ru
        r[active] = (1.0 - alpha) * ru / 2.0
        pushes[active] += 1
        # x(u) goes to every row of column u: y = A x
        lens = colptr[active + 1] - colptr[active]
        first = np.repeat(colptr[active] - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens)
        rows = rowidx[first + np.arange(int(lens.sum()))]
        r += np.bincount(rows, weights=np.repeat(xu, lens), minlength=n)
        steps += 1
    return p, r, steps, pushes, margin
