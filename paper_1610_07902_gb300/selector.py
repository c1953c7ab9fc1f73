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


def bfs_levels(colptr, rowidx, src):
    """Levels of a BFS from src (host, for building replay frontiers)."""
    import scipy.sparse as sp
    import scipy.sparse.csgraph as csg
    n = colptr.shape[0] - 1
    G = sp.csc_matrix((np.ones(rowidx.shape[0], np.int8), rowidx, colptr), shape=(n, n))
    d = csg.shortest_path(G.T, method="D", unweighted=True, indices=int(src))
    return np.where(np.isinf(d), -1, d).astype(np.int32)


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
        lev = bfs_levels(A.colptr, A.rowidx, src)
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
                opts = S.SPMSPV_MASK_COMPLEMENT | S.SPMSPV_SCHED_OPT(sched)
                fn = lambda: S.spmspv_run(Ad.handle, S.SPMSPV_MIN_SELECT2ND_I32, xi, xi, front.size, mk,
                                          opts, y_idx, y_val, cap, nz)
                fn()
                row[sched] = time_call(fn, reps)
            S.spmspv_run(Ad.handle, S.SPMSPV_MIN_SELECT2ND_I32, xi, xi, front.size, mk,
                         S.SPMSPV_MASK_COMPLEMENT | S.SPMSPV_WITH_FEATURES, y_idx, y_val, cap, nz)
            feats.append(S.spmspv_last_features(Ad.handle))
            v = ~np.isnan(row)
            targ.append(np.where(v, np.log2(np.where(v, row, 1.0)), 0.0))
            valid.append(v.astype(np.uint8))
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
    ("rmat16", ("rmat", 16, 11)), ("rmat18", ("rmat", 18, 12)), ("rmat20", ("rmat", 20, 13)),
    ("grid2d_512", ("grid", (512, 512, 1))), ("grid2d_1024", ("grid", (1024, 1024, 1))),
    ("grid3d_64", ("grid", (64, 64, 64))), ("grid3d_128", ("grid", (128, 128, 128))),
]


def training_graphs():
    import synth
    for name, spec in TRAINING_GRAPHS:
        if spec[0] == "rmat":
            yield name, synth.rmat(spec[1], seed=spec[2])
        else:
            yield name, synth.grid3d(*spec[1], 0.05, seed=3)


def main():
    import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--sources", type=int, default=2)
    ap.add_argument("--epochs", type=int, default=400)
    args = ap.parse_args()
    S.load()
    F, T, V = [], [], []
    t0 = time.time()
    last = None
    for name, A in training_graphs():
        Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
        f, t, v = collect(Ad, A, synth.sources(A.colptr, args.sources, seed=5))
        print("%-12s levels %4d  (%.0f s)" % (name, f.shape[0], time.time() - t0), file=sys.stderr)
        F.append(f), T.append(t), V.append(v)
        if last is not None:
            last.close()
        last = Ad
    F, T, V = np.concatenate(F), np.concatenate(T), np.concatenate(V)
    losses = train(last, F, T, V, epochs=args.epochs)
    params = S.spmspv_selector_get(last.handle)
    save(params, args.out, {"samples": int(F.shape[0]), "final_loss": float(losses[-1]),
                            "graphs": [g for g, _ in TRAINING_GRAPHS]})
    np.savez(os.path.splitext(args.out)[0] + "_data.npz", feats=F, target=T, valid=V)
    print("trained on %d levels, loss %.4f -> %.4f" % (F.shape[0], losses[0], losses[-1]),
          file=sys.stderr)


if __name__ == "__main__":
    main()
