"""Training data and training for the learned schedule selector.

The selector (csrc/selector.cu) is trained on timings the method generates
itself: every level of a BFS is replayed through spmspv_run under each of the
12 schedules (identical results, different kernels and tile/bucket sizes),
its device-side features are recorded, and the network is fitted to the log
run times with the library's own forward/backward kernels
(spmspv_selector_train).  Parameters are stored as JSON.

    python -m paper_1610_07902_gb300.selector --out weights.json
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np
import torch

from . import spmspv as S

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_weights.json")


def bfs_levels(Ad, src):
    """Levels of a BFS from src, computed by the library's own BFS (only used
    to build the frontiers that the timing replays)."""
    level, _, _ = Ad.bfs(int(src))
    return level.cpu().numpy()


def time_call(fn, reps):
    st = torch.cuda.current_stream()
    best = math.inf
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        fn()
        b.record(st)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def collect(Ad, A, sources, reps=3, max_levels=64, rng=None):
    """(features [N,6], log2 ms [N,12], valid [N,12]) from BFS level replays."""
    rng = rng or np.random.default_rng(0)
    can_pull = bool(Ad.flags & S.SPMSPV_CSC_PATTERN_SYMMETRIC)
    feats, targ, valid = [], [], []
    dev = Ad.colptr.device
    cap = A.m
    y_idx = torch.empty(cap, dtype=torch.int32, device=dev)
    y_val = torch.empty(cap, dtype=torch.int32, device=dev)
    nz = torch.zeros(1, dtype=torch.int32, device=dev)
    for src in sources:
        lev = bfs_levels(Ad, src)
        nl = int(lev.max()) + 1
        levels = list(range(nl))
        if len(levels) > max_levels:
            levels = sorted(rng.choice(nl, size=max_levels, replace=False).tolist())
        for L in levels:
            front = np.flatnonzero(lev == L).astype(np.int32)
            if front.size == 0:
                continue
            rng.shuffle(front)
            visited = ((lev >= 0) & (lev <= L)).astype(np.uint8)
            bits = np.packbits(np.pad(visited, (0, (-A.m) % 32)), bitorder="little").view("<u4")
            xi = torch.from_numpy(front).to(dev)
            mk = torch.from_numpy(bits.astype(np.uint32).view(np.int32)).to(dev)
            row = np.full(12, np.nan)
            for sched in range(12):
                if sched >= 6 and not can_pull:
                    continue
                # x(j) = j: the pull stops at a row's first frontier neighbour,
                # as inside the BFS loop the network's choices are used in
                opts = S.SPMSPV_MASK_COMPLEMENT | S.SPMSPV_X_IDS | S.SPMSPV_SCHED_OPT(sched)
                fn = lambda: S.spmspv_run(Ad.handle, S.SPMSPV_MIN_SELECT2ND_I32, xi, xi, front.size, mk,
                                          opts, y_idx, y_val, cap, nz)
                fn()
                row[sched] = time_call(fn, reps)
            S.spmspv_run(Ad.handle, S.SPMSPV_MIN_SELECT2ND_I32, xi, xi, front.size, mk,
                         S.SPMSPV_MASK_COMPLEMENT | S.SPMSPV_X_IDS | S.SPMSPV_WITH_FEATURES, y_idx, y_val, cap, nz)
            feats.append(S.spmspv_last_features(Ad.handle))
            v = ~np.isnan(row)
            targ.append(np.where(v, np.log2(np.where(v, row, 1.0)), 0.0))
            valid.append(v.astype(np.uint8))
    return (np.array(feats, np.float32), np.array(targ, np.float32), np.array(valid, np.uint8))


def plain_frontiers(n, count, rng):
    """`count` frontiers of log-uniform size in [1, n] (distinct ids, random order)."""
    import synth
    sizes = np.unique(np.maximum(1, np.floor(10 ** rng.uniform(0, np.log10(n), count))).astype(np.int64))
    return [synth.frontier(n, int(f), seed=int(rng.integers(1 << 30)), stream=2) for f in sizes]


def collect_plain(A, count=10, reps=3, rng=None):
    """(features, log2 ms, valid) from unmasked (+,*) products with values,
    x of log-uniform size: the calls a BFS level never looks like (no mask,
    up to every column), timed under every push schedule."""
    rng = rng or np.random.default_rng(1)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val)
    dev = Ad.colptr.device
    cap = A.m
    y_idx = torch.empty(cap, dtype=torch.int32, device=dev)
    y_val = torch.empty(cap, dtype=torch.float32, device=dev)
    nz = torch.zeros(1, dtype=torch.int32, device=dev)
    feats, targ, valid = [], [], []
    for xi_h, xv_h in plain_frontiers(A.n, count, rng):
        xi, xv = torch.from_numpy(xi_h).to(dev), torch.from_numpy(xv_h).to(dev)
        row = np.full(12, np.nan)
        for sched in range(6):
            fn = lambda: S.spmspv_run(Ad.handle, S.SPMSPV_PLUS_TIMES_F32, xi, xv, xi_h.size, None,
                                      S.SPMSPV_SCHED_OPT(sched), y_idx, y_val, cap, nz)
            fn()
            row[sched] = time_call(fn, reps)
        S.spmspv_run(Ad.handle, S.SPMSPV_PLUS_TIMES_F32, xi, xv, xi_h.size, None, S.SPMSPV_WITH_FEATURES,
                     y_idx, y_val, cap, nz)
        feats.append(S.spmspv_last_features(Ad.handle))
        v = ~np.isnan(row)
        targ.append(np.where(v, np.log2(np.where(v, row, 1.0)), 0.0))
        valid.append(v.astype(np.uint8))
    Ad.close()
    return (np.array(feats, np.float32), np.array(targ, np.float32), np.array(valid, np.uint8))


def train(Ad, feats, targ, valid, epochs=300, batch=64, lr=3e-3, seed=1):
    dev = Ad.colptr.device
    f = torch.from_numpy(np.ascontiguousarray(feats)).to(dev)
    t = torch.from_numpy(np.ascontiguousarray(targ)).to(dev)
    v = torch.from_numpy(np.ascontiguousarray(valid)).to(dev)
    return S.spmspv_selector_train(Ad.handle, f, t, v, feats.shape[0], epochs, batch, lr, seed)


def save(params, path=WEIGHTS, meta=None):
    with open(path, "w") as fh:
        json.dump({"nparam": int(len(params)), "params": [float(x) for x in params],
                   "meta": meta or {}}, fh)


def load(path=WEIGHTS):
    with open(path) as fh:
        d = json.load(fh)
    return np.array(d["params"], np.float32), d.get("meta", {})


TRAINING_GRAPHS = [
    ("rmat16", ("rmat", 16, 11)), ("rmat17", ("rmat", 17, 14)), ("rmat18", ("rmat", 18, 12)),
    ("rmat19", ("rmat", 19, 15)), ("rmat20", ("rmat", 20, 13)), ("rmat21", ("rmat", 21, 16)),
    ("grid2d_512", ("grid", (512, 512, 1))), ("grid2d_1024", ("grid", (1024, 1024, 1))),
    ("grid2d_2048", ("grid", (2048, 2048, 1))),
    ("grid3d_64", ("grid", (64, 64, 64))), ("grid3d_128", ("grid", (128, 128, 128))),
    ("grid3d_161", ("grid", (161, 161, 161))),
]

# held out from training: a larger R-MAT and a larger 3D grid
EVAL_GRAPHS = [("rmat23", ("rmat", 23, 21)), ("grid3d_320", ("grid", (320, 320, 320)))]
EVAL_GRAPHS_SMALL = [("rmat22", ("rmat", 22, 21)), ("grid3d_256", ("grid", (256, 256, 256)))]


def make_graph(spec, values=False):
    import synth
    if spec[0] == "rmat":
        return synth.rmat(spec[1], seed=spec[2], values=values)
    return synth.grid3d(*spec[1], 0.05, seed=3, values=values)


def training_graphs():
    for name, spec in TRAINING_GRAPHS:
        yield name, make_graph(spec)


def time_bfs(Ad, src, opts, reps=3):
    """Device time (ms) of one whole spmspv_bfs (graph-captured level loop)."""
    dev = Ad.colptr.device
    level = torch.empty(Ad.n, dtype=torch.int32, device=dev)
    parent = torch.empty(Ad.n, dtype=torch.int32, device=dev)
    nl = torch.zeros(1, dtype=torch.int32, device=dev)
    fn = lambda: S.spmspv_bfs(Ad.handle, int(src), level, parent, nl, opts)
    fn()
    return time_call(fn, reps), level, parent


def evaluate(Ad, A, sources, params, reps=3, max_levels=48, rng=None):
    """Held-out evaluation of the trained selector on one graph.

    Per call (replayed BFS levels): regret t/t_best - 1 of the schedule the
    network picks (t from the same table), of the AUTO call as run (network
    inference included) and of the fixed default schedule.  Per BFS: total
    device time under the default schedule, AUTO, and the best single fixed
    schedule (the autotuned fixed choice), with levels and parents checked
    identical across all of them.
    """
    rng = rng or np.random.default_rng(0)
    S.spmspv_selector_set(Ad.handle, params)
    default = S.spmspv_default_schedule(Ad.handle)
    dev = Ad.colptr.device
    cap = A.m
    y_idx = torch.empty(cap, dtype=torch.int32, device=dev)
    y_val = torch.empty(cap, dtype=torch.int32, device=dev)
    nz = torch.zeros(1, dtype=torch.int32, device=dev)
    pick_regret, auto_regret, fixed_regret, picks = [], [], [], []
    for src in sources:
        lev = bfs_levels(Ad, src)
        nl = int(lev.max()) + 1
        levels = list(range(nl))
        if len(levels) > max_levels:
            levels = sorted(rng.choice(nl, size=max_levels, replace=False).tolist())
        for L in levels:
            front = np.flatnonzero(lev == L).astype(np.int32)
            if front.size == 0:
                continue
            rng.shuffle(front)
            visited = ((lev >= 0) & (lev <= L)).astype(np.uint8)
            bits = np.packbits(np.pad(visited, (0, (-A.m) % 32)), bitorder="little").view("<u4")
            xi = torch.from_numpy(front).to(dev)
            mk = torch.from_numpy(bits.astype(np.uint32).view(np.int32)).to(dev)
            call = lambda o: (lambda: S.spmspv_run(Ad.handle, S.SPMSPV_MIN_SELECT2ND_I32, xi, xi,
                                                   front.size, mk,
                                                   S.SPMSPV_MASK_COMPLEMENT | S.SPMSPV_X_IDS | o,
                                                   y_idx, y_val, cap, nz))
            t = np.full(12, np.inf)
            for sched in range(12):
                fn = call(S.SPMSPV_SCHED_OPT(sched))
                fn()
                t[sched] = time_call(fn, reps)
            fa = call(S.SPMSPV_SCHED_AUTO)
            fa()
            ta = time_call(fa, reps)
            pick = S.spmspv_last_schedule(Ad.handle)
            best = t.min()
            picks.append(pick)
            pick_regret.append(t[pick] / best - 1)
            auto_regret.append(ta / best - 1)
            fixed_regret.append(t[default] / best - 1)
    q = lambda v: {"mean": float(np.mean(v)), "median": float(np.median(v)),
                   "p90": float(np.percentile(v, 90)), "max": float(np.max(v))}
    per_call = {"calls": len(picks), "picked_schedule": q(pick_regret),
                "auto_as_run": q(auto_regret), "fixed_default": q(fixed_regret),
                "pick_histogram": np.bincount(picks, minlength=12).tolist()}
    totals = {"fixed_default": 0.0, "auto": 0.0}
    per_sched = np.zeros(12)
    identical = True
    for src in sources:
        tf, lf, pf = time_bfs(Ad, src, S.SPMSPV_SCHED_OPT(default), reps)
        ta, la, pa = time_bfs(Ad, src, S.SPMSPV_SCHED_AUTO, reps)
        identical &= bool(torch.equal(lf, la) and torch.equal(pf, pa))
        totals["fixed_default"] += tf
        totals["auto"] += ta
        for sched in range(12):
            ts, ls, ps = time_bfs(Ad, src, S.SPMSPV_SCHED_OPT(sched), reps)
            identical &= bool(torch.equal(lf, ls) and torch.equal(pf, ps))
            per_sched[sched] += ts
    best_fixed = int(np.argmin(per_sched))
    totals.update({"best_fixed_schedule": best_fixed, "best_fixed": float(per_sched[best_fixed]),
                   "per_schedule": per_sched.tolist(), "sources": len(sources),
                   "identical_results": identical,
                   "auto_vs_fixed_default": totals["fixed_default"] / totals["auto"],
                   "auto_vs_best_fixed": float(per_sched[best_fixed]) / totals["auto"]})
    return {"per_call_regret": per_call, "bfs_total_ms": totals, "default_schedule": default}


def evaluate_plain(A, params, count=8, reps=3, rng=None):
    """Held-out evaluation on unmasked (+,*) products with values (x of
    log-uniform size): per call, the regret of the picked schedule and of the
    fixed default, and the time of AUTO as run against the fixed default."""
    rng = rng or np.random.default_rng(3)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val)
    S.spmspv_selector_set(Ad.handle, params)
    default = S.spmspv_default_schedule(Ad.handle)
    dev = Ad.colptr.device
    cap = A.m
    y_idx = torch.empty(cap, dtype=torch.int32, device=dev)
    y_val = torch.empty(cap, dtype=torch.float32, device=dev)
    nz = torch.zeros(1, dtype=torch.int32, device=dev)
    rows = []
    for xi_h, xv_h in plain_frontiers(A.n, count, rng):
        xi, xv = torch.from_numpy(xi_h).to(dev), torch.from_numpy(xv_h).to(dev)
        call = lambda o: (lambda: S.spmspv_run(Ad.handle, S.SPMSPV_PLUS_TIMES_F32, xi, xv, xi_h.size, None,
                                               o, y_idx, y_val, cap, nz))
        t = np.full(6, np.inf)
        for sched in range(6):
            fn = call(S.SPMSPV_SCHED_OPT(sched))
            fn()
            t[sched] = time_call(fn, reps)
        fa = call(S.SPMSPV_SCHED_AUTO)
        fa()
        ta = time_call(fa, reps)
        pick = S.spmspv_last_schedule(Ad.handle)
        rows.append({"nnz_x": int(xi_h.size), "pick": pick, "pick_regret": float(t[pick] / t.min() - 1),
                     "fixed_regret": float(t[default] / t.min() - 1),
                     "auto_vs_fixed_default": float(t[default] / ta)})
    Ad.close()
    return rows


def main_evaluate(args):
    import synth
    params, meta = load(args.weights)
    out = {"weights": os.path.basename(args.weights), "trained_on": meta.get("graphs"), "graphs": {}}
    for name, spec in (EVAL_GRAPHS_SMALL if args.small else EVAL_GRAPHS):
        t0 = time.time()
        A = make_graph(spec)
        Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
        r = evaluate(Ad, A, synth.sources(A.colptr, args.sources, seed=7), params)
        r.update({"n": int(A.n), "nnz": int(A.nnz)})
        Ad.close()
        del A
        r["plain_plus_times"] = evaluate_plain(make_graph(spec, values=True), params)
        out["graphs"][name] = r
        print("%-12s %s (%.0f s)" % (name, json.dumps(r["bfs_total_ms"]), time.time() - t0),
              file=sys.stderr)
        print("%-12s plain (+,*): %s" % (name, json.dumps(r["plain_plus_times"])), file=sys.stderr)
    with open(args.eval_out, "w") as fh:
        json.dump(out, fh, indent=1)


def main():
    import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--sources", type=int, default=2)
    ap.add_argument("--rmat-sources", type=int, default=0,
                    help="BFS sources per R-MAT training graph (default: --sources); an R-MAT search has a "
                         "few levels, a grid search hundreds")
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--evaluate", action="store_true",
                    help="evaluate --weights on the held-out graphs instead of training")
    ap.add_argument("--weights", default=WEIGHTS)
    ap.add_argument("--eval-out", default="selector_eval.json")
    ap.add_argument("--small", action="store_true", help="held-out graphs one size smaller")
    ap.add_argument("--plain-calls", type=int, default=0,
                    help="also train on this many unmasked (+,*) calls per graph (default: BFS levels only)")
    args = ap.parse_args()
    S.load()
    if args.evaluate:
        main_evaluate(args)
        return
    F, T, V = [], [], []
    t0 = time.time()
    last = None
    for (name, spec), (_, A) in zip(TRAINING_GRAPHS, training_graphs()):
        Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
        nsrc = args.rmat_sources if (spec[0] == "rmat" and args.rmat_sources) else args.sources
        f, t, v = collect(Ad, A, synth.sources(A.colptr, nsrc, seed=5))
        fp, tp, vp = (collect_plain(make_graph(spec, values=True), count=args.plain_calls) if args.plain_calls
                      else (np.zeros((0, 6), np.float32), np.zeros((0, 12), np.float32), np.zeros((0, 12), np.uint8)))
        print("%-12s levels %4d, plain calls %3d  (%.0f s)" % (name, f.shape[0], fp.shape[0], time.time() - t0),
              file=sys.stderr)
        F += [f, fp]
        T += [t, tp]
        V += [v, vp]
        if last is not None:
            last.close()
        last = Ad
    F, T, V = np.concatenate(F), np.concatenate(T), np.concatenate(V)
    losses = train(last, F, T, V, epochs=args.epochs)
    params = S.spmspv_selector_get(last.handle)
    save(params, args.out, {"samples": int(F.shape[0]), "final_loss": float(losses[-1]),
                            "sources": args.sources, "rmat_sources": args.rmat_sources or args.sources,
                            "sample_kinds": ("BFS level replays and unmasked (+,*) calls" if args.plain_calls
                                             else "BFS level replays"),
                            "graphs": [g for g, _ in TRAINING_GRAPHS]})
    np.savez(os.path.splitext(args.out)[0] + "_data.npz", feats=F, target=T, valid=V)
    print("trained on %d calls, loss %.4f -> %.4f" % (F.shape[0], losses[0], losses[-1]),
          file=sys.stderr)


if __name__ == "__main__":
    main()
