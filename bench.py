"""Benchmark of the GB300 SpMSpV path (one JSON line on rank 0).

Workload (the headline configuration): R-MAT scale 22, edge factor 16,
a/b/c/d = .57/.19/.19/.05, symmetrised, self-loops and duplicates removed,
int32 CSC, float32 values uniform(0,1), seed 1; x = 10^6 distinct uniform
random indices with uniform(0,1) values; semiring (+,*) in float32.
One step = one SpMSpV y <- A x through the C ABI (work scan, expand/scatter,
bucket merge); the L2 cache is flushed (a 256 MiB write) before every timed
step.  GTEPS = products (the sum of the selected column lengths) / second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (launched by torchrun) every rank runs an independent replica of
the workload on its own GPU: the SpMSpV does not shard, so the value is the
products of all ranks over the slowest rank's time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SpMSpV GTEPS & % HBM roofline at R-MAT s22; learned/batched vs plain BFS time"
WORKLOAD = "rmat22_ef16_f1e6_plus_times_f32"
SCALE, EDGE_FACTOR, SEED, F = 22, 16, 1, 1_000_000


def kernels_hash():
    """First 16 hex digits of the SHA-256 of the kernel sources the capture
    covers (kernels.cu and the headers it includes)."""
    import hashlib
    h = hashlib.sha256()
    base = os.path.join(ROOT, "paper_1610_07902_gb300", "csrc")
    for name in ("kernels.cu", "expand_dev.cuh", "spmspv_internal.cuh", "device_util.cuh",
                 "selector_dev.cuh"):
        with open(os.path.join(base, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic(kernel):
    """DRAM bytes per unit of `kernel` from a committed ncu summary under
    profiles/ whose capture was of these exact kernel sources: a line
    'traffic: <kernel> <bytes per unit> bytes per <unit> (sources <hash>)'.
    None when no summary matches the current sources."""
    import glob
    import re
    want = kernels_hash()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path):
            m = re.search(r"traffic: (\S+) ([0-9.]+) bytes per (\w+) \(sources ([0-9a-f]+)\)", line)
            if m and m.group(1) == kernel and m.group(4) == want:
                return float(m.group(2)), os.path.basename(path)
    return None, None


NOMINAL_HBM_GBS = 7900.0  # nominal HBM3e bandwidth of the part, a second denominator


def host_cpu():
    """Host threads and CPU model (for the oracle baseline)."""
    import platform
    model = platform.processor() or platform.machine()
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return os.cpu_count(), model


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def make_inputs(scale=SCALE, f=F):
    import synth
    A = synth.rmat(scale, EDGE_FACTOR, seed=SEED)
    x_idx, x_val = synth.frontier(A.n, f, seed=1, stream=2)
    return A, x_idx, x_val


def compulsory_bytes(f, W, ny):
    """(+,*) fp32: x (8f) + two column pointers per x entry (8f) + row id and
    value per product (8W) + y (8 nnz(y))."""
    return 8 * f + 8 * f + 8 * W + 8 * ny


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the GPU is busy."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        sel = []
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            sel = ["-i", vis.split(",")[device_index]]
        else:
            sel = ["-i", str(device_index)]
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "50"] + sel,
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:]))
            except ValueError:
                continue
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [r[0] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2])
                          if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def time_oracle(A, x_idx, x_val, budget_s=10.0):
    """The oracle as it stands, single-threaded, on a bounded sample."""
    import oracle
    W_total, t_total, calls = 0, 0.0, 0
    per_call = []
    while t_total < budget_s or calls == 0:
        t0 = time.perf_counter()
        r = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, oracle.PLUS_TIMES, x_idx, x_val,
                          with_absum=False)
        dt = time.perf_counter() - t0
        t_total += dt
        per_call.append(dt)
        W_total += r.nmult
        calls += 1
        if calls >= 20:
            break
    time_oracle.median_s = float(np.median(per_call))
    return W_total / t_total / 1e9, calls, t_total


def replica_summary(t_ms, products_per_step, steps, world, device):
    """Replicas only: every rank runs the whole workload on its own GPU.  The
    job time is the slowest rank's (barrier, then the maximum over ranks) and
    the value is the products of all ranks over that time, in GTEPS."""
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        tt = torch.tensor([t_ms], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms = float(tt.item())
    return t_ms, products_per_step * steps * world / (t_ms * 1e-3) / 1e9


def _events_ms(fn, stream, reps=1):
    import torch
    best = float("inf")
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def selector_params():
    from paper_1610_07902_gb300 import selector
    try:
        return selector.load()[0]
    except (OSError, ValueError, KeyError):
        return None


def bench_bfs(S, A, dev, stream, name, sources, params, pt_frontiers=False):
    """BFS under the plain fixed schedule and under the learned selector (AUTO),
    one graph-captured level loop per search, levels and parents compared."""
    import torch
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC,
                     device=dev)
    deg = torch.diff(Ad.colptr.long())
    level = torch.empty(A.n, dtype=torch.int32, device=dev)
    parent = torch.empty(A.n, dtype=torch.int32, device=dev)
    level2 = torch.empty_like(level)
    parent2 = torch.empty_like(parent)
    nl = torch.zeros(1, dtype=torch.int32, device=dev)
    default = S.spmspv_default_schedule(Ad.handle)
    fixed = S.SPMSPV_SCHED_OPT(default)
    if params is not None:
        S.spmspv_selector_set(Ad.handle, params)
    t_fixed = t_auto = t_rule = 0.0
    work = 0
    reached = 0
    levels = []
    same = True
    for src in sources:
        run = lambda o, lv, pa: S.spmspv_bfs(Ad.handle, int(src), lv, pa, nl, o, stream)
        run(fixed, level, parent)
        t_fixed += _events_ms(lambda: run(fixed, level, parent), stream, 2)
        levels.append(int(nl.item()))
        work += int(deg[level >= 0].sum().item())
        reached += int((level >= 0).sum().item())
        # the direction-optimizing rule (two fixed thresholds), the learned selector's baseline
        run(S.SPMSPV_SCHED_RULE, level2, parent2)
        t_rule += _events_ms(lambda: run(S.SPMSPV_SCHED_RULE, level2, parent2), stream, 2)
        same &= bool(torch.equal(level, level2) and torch.equal(parent, parent2))
        if params is not None:
            run(S.SPMSPV_SCHED_AUTO, level2, parent2)
            t_auto += _events_ms(lambda: run(S.SPMSPV_SCHED_AUTO, level2, parent2), stream, 2)
            same &= bool(torch.equal(level, level2) and torch.equal(parent, parent2))
    # compulsory bytes of the (select2nd, min) searches, without the mask reads:
    # every reached vertex is one x entry (8 B) with two column pointers (8 B),
    # one y entry (8 B) and a level and a parent (8 B); 4 B of row id per product
    bfs_bytes = 32 * reached + 4 * work
    peak, _ = load_peaks()
    out = {"graph": name, "n": A.n, "nnz": A.nnz, "sources": len(sources),
           "levels_max": max(levels), "products": work, "default_schedule": default,
           "fixed_ms": t_fixed, "fixed_gteps": work / (t_fixed * 1e-3) / 1e9,
           "compulsory_bytes_min_semiring": bfs_bytes,
           "fixed_path_frac": bfs_bytes / (t_fixed * 1e-3) / 1e9 / peak}
    out.update({"rule_ms": t_rule, "rule_speedup": t_fixed / t_rule, "identical_results": same})
    if params is not None:
        out.update({"auto_ms": t_auto, "auto_gteps": work / (t_auto * 1e-3) / 1e9,
                    "auto_speedup": t_fixed / t_auto, "auto_vs_rule": t_rule / t_auto})
    if pt_frontiers:
        # (+,*) float32 SpMSpV on every frontier of the last search (level sets
        # from the device BFS, host-side split), one call per level
        lv = level.cpu().numpy()
        fr = [torch.from_numpy(np.flatnonzero(lv == L).astype(np.int32)).to(dev)
              for L in range(int(lv.max()) + 1)]
        xv = [torch.rand(f.shape[0], device=dev) for f in fr]
        cap = min(A.m, A.nnz)
        yi = torch.empty(cap, dtype=torch.int32, device=dev)
        yv = torch.empty(cap, dtype=torch.float32, device=dev)
        nz = torch.zeros(1, dtype=torch.int32, device=dev)
        pw = int(sum(deg[f.long()].sum().item() for f in fr))

        def all_levels():
            for f, v in zip(fr, xv):
                S.spmspv_run(Ad.handle, S.SPMSPV_PLUS_TIMES_F32, f, v, f.shape[0], None, 0, yi, yv,
                             cap, nz, stream)
        all_levels()
        t = _events_ms(all_levels, stream, 2)
        out["plus_times_per_frontier"] = {"calls": len(fr), "products": pw, "ms": t,
                                          "gteps": pw / (t * 1e-3) / 1e9,
                                          "us_per_call": 1e3 * t / len(fr)}
        # the same products as one batched launch (autotuned lanes)
        B = len(fr)
        x_cnt = np.array([f.shape[0] for f in fr], np.int32)
        x_off = np.concatenate([[0], np.cumsum(x_cnt)[:-1]]).astype(np.int32)
        y_cap = np.array([max(1, int(deg[f.long()].sum().item())) for f in fr], np.int64)
        y_off = np.concatenate([[0], np.cumsum(y_cap)[:-1]])
        td = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        xi_all, xv_all = torch.cat(fr), torch.cat(xv)
        yi_all = torch.empty(int(y_cap.sum()), dtype=torch.int32, device=dev)
        yv_all = torch.empty(int(y_cap.sum()), dtype=torch.float32, device=dev)
        nz_all = torch.zeros(B, dtype=torch.int32, device=dev)
        d_off, d_cnt = td(x_off), td(x_cnt)
        d_yoff, d_ycap = td(y_off.astype(np.int32)), td(y_cap.astype(np.int32))

        def batched():
            S.spmspv_run_batched(Ad.handle, S.SPMSPV_PLUS_TIMES_F32, B, d_off, d_cnt, xi_all, xv_all,
                                 None, 0, 0, d_yoff, d_ycap, yi_all, yv_all, nz_all, 0, stream)
        batched()  # tunes on first use
        tb = _events_ms(batched, stream, 2)
        tuned = S.spmspv_last_tuned(Ad.handle)
        nzb = nz_all.cpu().numpy()
        same = True
        for b in range(0, B, max(1, B // 24)):  # spot check against single calls
            S.spmspv_run(Ad.handle, S.SPMSPV_PLUS_TIMES_F32, fr[b], xv[b], fr[b].shape[0], None,
                         S.SPMSPV_SORTED_OUT, yi, yv, cap, nz, stream)
            k = int(nz.item())
            o = int(y_off[b])
            same &= k == int(nzb[b]) and torch.equal(yi[:k], yi_all[o:o + k])
        out["plus_times_per_frontier"].update({
            "batched_ms": tb, "batched_gteps": pw / (tb * 1e-3) / 1e9, "batched_speedup": t / tb,
            "batched_lanes": tuned[0], "batched_schedule": tuned[1], "batched_identical_index_sets": same})
    Ad.close()
    return out


def graph_us_per_call(call, stream, reps=100):
    """GPU time per call with the host out of the way: `reps` calls captured
    into one CUDA graph (call(stream) launches on the capture stream), the
    graph replayed and timed with events.  None if the capture fails."""
    import torch
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            cs = torch.cuda.current_stream()
            for _ in range(reps):
                call(cs)
        g.replay()
        torch.cuda.synchronize()
        t = _events_ms(g.replay, stream, 3)
        del g
        return 1e3 * t / reps
    except Exception:  # capture not possible here: report the host-launched figure only
        torch.cuda.synchronize()
        return None


def bench_er(S, dev, stream):
    """The Sec. II-A model: Erdos-Renyi m = n = 65,536 with 16/65,536 density
    (directed, self loops allowed, values uniform(0,1), seed 1); x of 655
    entries (seed 1 stream 2).  Latency-bound: microseconds per call and
    GTEPS, back-to-back host-launched calls (the whole problem sits in L2)."""
    import torch
    import synth
    A = synth.erdos_renyi(65536, 16.0, seed=1)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val, device=dev)
    xi_, xv_ = synth.frontier(A.n, 655, seed=1, stream=2)
    xi, xv = torch.from_numpy(xi_).to(dev), torch.from_numpy(xv_).to(dev)
    cap = min(A.m, A.nnz)
    yi = torch.empty(cap, dtype=torch.int32, device=dev)
    yv = torch.empty(cap, dtype=torch.float32, device=dev)
    nz = torch.zeros(1, dtype=torch.int32, device=dev)
    run = lambda: S.spmspv_run(Ad.handle, S.SPMSPV_PLUS_TIMES_F32, xi, xv, 655, None, S.SPMSPV_SORTED_OUT,
                               yi, yv, cap, nz, stream)
    for _ in range(10):
        run()
    reps = 500
    t = _events_ms(lambda: [run() for _ in range(reps)], stream, 1) / reps
    W = S.spmspv_last_work(Ad.handle)
    tg = graph_us_per_call(lambda cs: S.spmspv_run(Ad.handle, S.SPMSPV_PLUS_TIMES_F32, xi, xv, 655, None,
                                                    S.SPMSPV_SORTED_OUT, yi, yv, cap, nz, cs), stream)
    out = {"m": A.m, "nnz": int(A.nnz), "nnz_x": 655, "products": W, "nnz_y": int(nz.item()),
           "us_per_call": 1e3 * t, "gteps": W / (t * 1e-3) / 1e9, "graph_us_per_call": tg,
           "status": S.spmspv_device_status(Ad.handle)}
    Ad.close()
    return out


def bench_cc(S, A, dev, stream):
    """Connected components of the headline graph (label propagation, one
    SpMSpV round per graph iteration, all rounds in one graph launch); the
    labels are checked by the properties every correct answer has (label[v]
    <= v, labels are their own labels, every edge joins equal labels)."""
    import torch
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC,
                     device=dev)
    labels = torch.empty(A.n, dtype=torch.int32, device=dev)
    rounds = torch.zeros(1, dtype=torch.int32, device=dev)
    run = lambda: S.spmspv_cc(Ad.handle, labels, rounds, 0, stream)
    run()
    t = _events_ms(run, stream, 3)
    lab = labels.long()
    col = torch.repeat_interleave(torch.arange(A.n, device=dev), torch.diff(Ad.colptr.long()))
    valid = bool((lab <= torch.arange(A.n, device=dev)).all() and (lab[lab] == lab).all()
                 and (lab[Ad.rowidx.long()] == lab[col]).all())
    comps = int((lab == torch.arange(A.n, device=dev)).sum().item())
    Ad.close()
    return {"ms": t, "rounds": int(rounds.item()), "components": comps, "labels_valid": valid}


def bench_mis(S, A, dev, stream):
    """Maximal independent set of the headline graph (Luby's rounds with a
    seeded random permutation as priorities, two SpMSpVs per round, all rounds
    in one graph launch).  Checked by the properties that single out the
    greedy set in priority order: no edge joins two members, and every
    non-member has a member neighbour of smaller priority."""
    import torch
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC,
                     device=dev)
    g = torch.Generator(device="cpu").manual_seed(7)
    prio = torch.randperm(A.n, generator=g).to(torch.int32).to(dev)
    in_set = torch.empty(A.n, dtype=torch.int32, device=dev)
    rounds = torch.zeros(1, dtype=torch.int32, device=dev)
    run = lambda: S.spmspv_mis(Ad.handle, prio, in_set, rounds, 0, stream)
    run()
    t = _events_ms(run, stream, 3)
    mem = in_set.bool()
    col = torch.repeat_interleave(torch.arange(A.n, device=dev), torch.diff(Ad.colptr.long()))
    row = Ad.rowidx.long()
    off = row != col
    independent = not bool((mem[row] & mem[col] & off).any())
    big = torch.iinfo(torch.int64).max
    p64 = prio.long()
    src = torch.where(mem[col] & off, p64[col], torch.full_like(p64[col], big))
    best = torch.full((A.n,), big, dtype=torch.int64, device=dev).scatter_reduce(0, row, src, "amin")
    dominated = bool(((best < p64) | mem).all())
    out = {"ms": t, "rounds": int(rounds.item()), "size": int(mem.sum().item()),
           "independent": independent, "each_nonmember_has_smaller_member_neighbour": dominated}
    del col, row, off, src, best
    Ad.close()
    return out


def bench_mcm(S, A, dev, stream):
    """Maximum matching between the rows and the columns of the headline
    matrix (phases of multi-source alternating BFS, one SpMSpV per level, all
    in one graph launch).  The matching is checked for validity here (mates
    agree, matched pairs are edges); that it is maximum is checked against the
    reference's cardinality in the tests, at sizes the reference finishes."""
    import torch
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None, device=dev)
    mate_r = torch.empty(A.m, dtype=torch.int32, device=dev)
    mate_c = torch.empty(A.n, dtype=torch.int32, device=dev)
    card = torch.zeros(1, dtype=torch.int32, device=dev)
    phases = torch.zeros(1, dtype=torch.int32, device=dev)
    run = lambda: S.spmspv_mcm(Ad.handle, mate_r, mate_c, card, phases, 0, stream)
    run()
    t = _events_ms(run, stream, 2)
    mc = mate_c.long()
    matched = torch.nonzero(mc >= 0).flatten()
    rows = mc[matched]
    agree = bool((mate_r.long()[rows] == matched).all()) and int((mate_r >= 0).sum()) == matched.numel()
    # a matched pair (i, j) is an edge: i lies in column j's row list
    cp = Ad.colptr.long()
    ri = Ad.rowidx.long()
    lo, hi = cp[matched], cp[matched + 1]
    key = matched * A.m + rows
    col = torch.repeat_interleave(torch.arange(A.n, device=dev), torch.diff(cp))
    edges = torch.sort(col * A.m + ri).values
    pos = torch.searchsorted(edges, key).clamp(max=edges.numel() - 1)
    edges_ok = bool((edges[pos] == key).all()) and bool((hi > lo).all())
    out = {"ms": t, "phases": int(phases.item()), "cardinality": int(card.item()),
           "matched_pairs_found": int(matched.numel()), "mates_agree": agree,
           "pairs_are_edges": edges_ok,
           "status": S.spmspv_device_status(Ad.handle)}
    del col, edges, pos, key, cp, ri
    Ad.close()
    return out


def bench_sorted_x(S, A, Ad, dev, stream, flush, y_idx, y_val, cap, nnz_y):
    """The sorted-versus-unsorted study of Sec. IV-B (Fig. 2 there: x with 10K
    and 2.5M nonzeros) on the headline matrix: x in random order, the same x
    sorted by the caller, and x in random order sorted on the device first
    (SPMSPV_SORT_X, the sort inside the timed call).  y is ascending in every
    case (the bucket order gives it for free).  Median of 9 calls, L2 flushed
    before each."""
    import torch
    import synth
    out = {}
    for fs in (10_000, 2_500_000):
        xi, xv = synth.frontier(A.n, fs, seed=5, stream=2)
        order = np.argsort(xi, kind="stable")
        variants = {
            "random_order": (xi, xv, 0),
            "sorted_by_caller": (xi[order], xv[order], 0),
            "device_presort": (xi, xv, S.SPMSPV_SORT_X),
        }
        res = {}
        nz = {}
        for name, (a, v, extra) in variants.items():
            dxi, dxv = torch.from_numpy(np.ascontiguousarray(a)).to(dev), torch.from_numpy(np.ascontiguousarray(v)).to(dev)
            run = lambda: S.spmspv_run(Ad.handle, S.SPMSPV_PLUS_TIMES_F32, dxi, dxv, fs, None,
                                       S.SPMSPV_SORTED_OUT | extra, y_idx, y_val, cap, nnz_y, stream)
            run()
            times = []
            for _ in range(9):
                flush.zero_()
                times.append(_events_ms(run, stream, 1))
            res[name + "_ms"] = float(np.median(times))
            nz[name] = int(nnz_y.item())
        res["products"] = S.spmspv_last_work(Ad.handle)
        res["same_nnz_y"] = len(set(nz.values())) == 1
        res["status"] = S.spmspv_device_status(Ad.handle)
        res["sorted_by_caller_vs_random"] = res["random_order_ms"] / res["sorted_by_caller_ms"]
        res["device_presort_vs_random"] = res["random_order_ms"] / res["device_presort_ms"]
        out["nnz_x_%d" % fs] = res
    return out


def bench_dcsc(S, dev, stream, flush):
    """A hypersparse block of the kind a 2D distribution hands each process
    (Sec. II-C): m = 2^22 rows, n = 2^25 columns of which nzc = 2^20 hold
    entries (16 on average), stored as DCSC and, for comparison, as CSC.  x
    with 10^6 ids uniform over all n columns (about 3% stored) and with 10^5
    ids among the stored columns.  Median of 9 calls, L2 flushed before each."""
    import torch
    m, n, nzc = 1 << 22, 1 << 25, 1 << 20
    rng = np.random.default_rng(17)
    cols = np.sort(rng.choice(n, size=nzc, replace=False)).astype(np.int64)
    d = rng.integers(1, 32, size=nzc)
    key = np.unique(np.repeat(cols, d) * m + rng.integers(0, m, size=int(d.sum())))
    col, row = key // m, (key % m).astype(np.int32)
    del key
    deg = np.bincount(col, minlength=n)
    del col
    colptr = np.concatenate([[0], np.cumsum(deg)]).astype(np.int32)
    jc = np.flatnonzero(deg > 0).astype(np.int32)
    cp = np.concatenate([[0], np.cumsum(deg[jc])]).astype(np.int32)
    val = rng.random(row.shape[0], dtype=np.float32)
    nnz = int(row.shape[0])
    Ac = S.CscMatrix(m, n, colptr, row, val, device=dev)
    Ad = S.DcscMatrix(m, n, jc, cp, row, val, device=dev)
    cap = m
    yi = torch.empty(cap, dtype=torch.int32, device=dev)
    yv = torch.empty(cap, dtype=torch.float32, device=dev)
    nz = torch.zeros(1, dtype=torch.int32, device=dev)
    out = {"m": m, "n": n, "nzc": int(jc.shape[0]), "nnz": nnz,
           "column_index_bytes": {"csc_colptr": 4 * (n + 1),
                                  "dcsc_jc_cp_aux": 4 * (2 * int(jc.shape[0]) + 1) + 4 * (int(jc.shape[0]) + 2)}}
    for name, xi_, f in (("uniform_over_n", rng.choice(n, size=1_000_000, replace=False), 1_000_000),
                         ("stored_columns", rng.choice(jc, size=100_000, replace=False), 100_000)):
        xi = torch.from_numpy(xi_.astype(np.int32)).to(dev)
        xv = torch.from_numpy(rng.random(f, dtype=np.float32)).to(dev)
        res = {}
        ys = []
        for hname, H in (("csc", Ac), ("dcsc", Ad)):
            run = lambda: S.spmspv_run(H.handle, S.SPMSPV_PLUS_TIMES_F32, xi, xv, f, None,
                                       S.SPMSPV_SORTED_OUT, yi, yv, cap, nz, stream)
            run()
            times = []
            for _ in range(9):
                flush.zero_()
                times.append(_events_ms(run, stream, 1))
            res[hname + "_ms"] = float(np.median(times))
            res["products"] = S.spmspv_last_work(H.handle)
            k = int(nz.item())
            ys.append((yi[:k].cpu().numpy().copy(), yv[:k].cpu().numpy().copy()))
            res[hname + "_status"] = S.spmspv_device_status(H.handle)
        res["same_y"] = bool(np.array_equal(ys[0][0], ys[1][0]) and
                             np.allclose(ys[0][1], ys[1][1], rtol=1e-5, atol=0))
        out[name] = res
    Ac.close()
    Ad.close()
    return out


def product_form(m, W, buckets_only):
    """Which form the library runs a (+,*) call in (the device's rule): the
    direct form from 2m products on (m <= 2^24), else the bucketed one."""
    return "direct" if not buckets_only and m <= (1 << 24) and W >= 2 * m else "bucketed"


def stage_roofline(S, form, F_, W, ny, stage_avg):
    """Stage names, the dominant stage's kernel, its captured traffic and its
    algorithmic HBM bytes: 16 B per x entry (scan), 8 B per product (row id and
    value read by the expand step; in the direct form its adds stay in L2),
    8 B per y entry (merge / compaction)."""
    if form == "direct":
        names = {S.SPMSPV_STAGE_SCAN: "work_scan", S.SPMSPV_STAGE_SCATTER: "expand_reduce",
                 S.SPMSPV_STAGE_MERGE: "compact"}
        knames = {S.SPMSPV_STAGE_SCAN: "k1_work_scan", S.SPMSPV_STAGE_SCATTER: "k2_expand_scatter[direct]",
                  S.SPMSPV_STAGE_MERGE: "k3_bucket_merge[direct]"}
    else:
        names = {S.SPMSPV_STAGE_SCAN: "work_scan", S.SPMSPV_STAGE_SCATTER: "expand_scatter",
                 S.SPMSPV_STAGE_MERGE: "bucket_merge"}
        knames = {S.SPMSPV_STAGE_SCAN: "k1_work_scan", S.SPMSPV_STAGE_SCATTER: "k2_expand_scatter",
                  S.SPMSPV_STAGE_MERGE: "k3_bucket_merge"}
    alg = {S.SPMSPV_STAGE_SCAN: 16 * F_, S.SPMSPV_STAGE_SCATTER: 8 * W, S.SPMSPV_STAGE_MERGE: 8 * ny}
    units = {S.SPMSPV_STAGE_SCAN: F_, S.SPMSPV_STAGE_SCATTER: W, S.SPMSPV_STAGE_MERGE: W}
    dom = max(names, key=lambda s: stage_avg[s])
    achieved = alg[dom] / (stage_avg[dom] * 1e-3) / 1e9
    per_unit, traffic_src = captured_traffic(knames[dom])
    return names, knames[dom], per_unit, traffic_src, units, alg, dom, achieved


def bench_bucketed_form(S, Ad, xi, xv, F_, y_idx, y_val, cap, nnz_y, stream, flush, peak, steps=100):
    """The headline product in the bucketed form (SPMSPV_BUCKETS_ONLY): the
    paper's row-range buckets and shared-memory SPA at every size."""
    import torch
    opts = S.SPMSPV_SORTED_OUT | S.SPMSPV_BUCKETS_ONLY

    def step():
        S.spmspv_run(Ad.handle, S.SPMSPV_PLUS_TIMES_F32, xi, xv, F_, None, opts, y_idx, y_val, cap, nnz_y,
                     stream)
    for _ in range(5):
        flush.zero_()
        step()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    W = S.spmspv_last_work(Ad.handle)
    ny = int(nnz_y.item())
    S.spmspv_profile_begin(Ad.handle)
    for _ in range(50):
        flush.zero_()
        step()
    stage_ms, ncalls = S.spmspv_profile_end(Ad.handle)
    stage_avg = [v / ncalls for v in stage_ms]
    names, kname, per_unit, src, units, alg, dom, achieved = stage_roofline(S, "bucketed", F_, W, ny, stage_avg)
    return {"ms_per_step": ms, "gteps": W / (ms * 1e-3) / 1e9,
            "stages_ms": {names[s]: stage_avg[s] for s in names},
            "roofline": {"kernel": kname, "achieved": achieved, "peak": peak, "frac": achieved / peak,
                         "traffic": per_unit * units[dom] if per_unit else None},
            "path_frac": compulsory_bytes(F_, W, ny) / (ms * 1e-3) / 1e9 / peak}


def bench_batched(S, dev, stream, B=256):
    """256 frontiers on R-MAT s20 in one batched launch (autotuned) against
    256 sequential plain calls; multi-source BFS and ACL the same way."""
    import torch
    import synth
    A = synth.rmat(20, EDGE_FACTOR, seed=4)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val, device=dev)
    rng = np.random.default_rng(4)
    sizes = np.maximum(1, np.floor(10 ** rng.uniform(0, 5, B))).astype(np.int64)
    fronts = [synth.frontier(A.n, int(f), seed=100 + b, stream=2) for b, f in enumerate(sizes)]
    x_cnt = sizes.astype(np.int32)
    x_off = np.concatenate([[0], np.cumsum(x_cnt)[:-1]]).astype(np.int32)
    td = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    xi_all = td(np.concatenate([f[0] for f in fronts]))
    xv_all = td(np.concatenate([f[1] for f in fronts]))
    y_off = (np.arange(B, dtype=np.int64) * A.m).astype(np.int64)
    ycap = A.m
    yi = torch.empty(B * ycap, dtype=torch.int32, device=dev)
    yv = torch.empty(B * ycap, dtype=torch.float32, device=dev)
    nz = torch.zeros(B, dtype=torch.int32, device=dev)
    d_off, d_cnt = td(x_off), td(x_cnt)
    d_yoff, d_ycap = td(y_off.astype(np.int32)), td(np.full(B, ycap, np.int32))

    def batched():
        S.spmspv_run_batched(Ad.handle, S.SPMSPV_PLUS_TIMES_F32, B, d_off, d_cnt, xi_all, xv_all, None,
                             0, 0, d_yoff, d_ycap, yi, yv, nz, 0, stream)
    batched()  # tunes on first use (the persistent form under every push schedule)
    t_b = _events_ms(batched, stream, 3)
    tuned = S.spmspv_last_tuned(Ad.handle)
    phases, waves = S.spmspv_batched_phase_times(Ad.handle)

    def lanes16():
        S.spmspv_run_batched(Ad.handle, S.SPMSPV_PLUS_TIMES_F32, B, d_off, d_cnt, xi_all, xv_all, None,
                             0, S.SPMSPV_SCHED_OPT(tuned[1]), d_yoff, d_ycap, yi, yv, nz, 16, stream)
    lanes16()
    t_l = _events_ms(lanes16, stream, 3)
    batched()
    nz_b = nz.cpu().numpy().copy()
    yi_b = yi.cpu().numpy()
    yv_b = yv.cpu().numpy()
    views = [(xi_all[x_off[b]:x_off[b] + x_cnt[b]], xv_all[x_off[b]:x_off[b] + x_cnt[b]],
              yi[b * ycap:(b + 1) * ycap], yv[b * ycap:(b + 1) * ycap], nz[b:b + 1]) for b in range(B)]

    def sequential():
        for b in range(B):
            a, v, oi, ov, on = views[b]
            S.spmspv_run(Ad.handle, S.SPMSPV_PLUS_TIMES_F32, a, v, int(x_cnt[b]), None,
                         S.SPMSPV_SORTED_OUT, oi, ov, ycap, on, stream)
    sequential()
    t_s = _events_ms(sequential, stream, 3)
    nz_s = nz.cpu().numpy()
    same_idx = bool((nz_s == nz_b).all())
    rel = 0.0
    yi_s, yv_s = yi.cpu().numpy(), yv.cpu().numpy()
    for b in range(B):
        o, c = b * ycap, int(nz_s[b])
        same_idx &= bool((yi_s[o:o + c] == yi_b[o:o + c]).all())
        d = np.abs(yv_s[o:o + c] - yv_b[o:o + c]) / np.maximum(np.abs(yv_s[o:o + c]), 1e-30)
        rel = max(rel, float(d.max()) if c else 0.0)
    W = int(sum(int(np.diff(A.colptr)[f[0]].sum()) for f in fronts))
    out = {"graph": "rmat s20 ef16 seed 4", "B": B, "nnz_x_loguniform": [1, 100000],
           "products": W,
           "spmspv": {"batched_ms": t_b, "sequential_ms": t_s, "speedup": t_s / t_b,
                      "batched_gteps": W / (t_b * 1e-3) / 1e9, "tuned_lanes": tuned[0],
                      "tuned_schedule": tuned[1], "form": "persistent" if tuned[0] == 0 else "lanes",
                      "phases_ms": dict(zip(["scan", "plan", "tile_starts", "expand", "merge", "launch",
                                             "direct_expand", "direct_compact"],
                                            [round(float(v), 4) for v in phases])),
                      "waves": waves, "lanes16_ms": t_l, "lanes16_gteps": W / (t_l * 1e-3) / 1e9,
                      "identical_index_sets": same_idx, "max_rel_value_diff": rel}}
    del yi, yv
    Ad.close()

    # multi-source BFS vs 256 sequential single-source BFS (fixed schedule)
    Ap = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None, flags=S.SPMSPV_CSC_SYMMETRIC, device=dev)
    srcs = synth.sources(A.colptr, B, seed=5).astype(np.int32)
    ds = td(srcs)
    lv = torch.empty(B * A.n, dtype=torch.int32, device=dev)
    pa = torch.empty(B * A.n, dtype=torch.int32, device=dev)
    ms = lambda: S.spmspv_msbfs(Ap.handle, B, ds, lv, pa, None, 0, 0, stream)
    ms()
    t_ms = _events_ms(ms, stream, 2)
    tuned = S.spmspv_last_tuned(Ap.handle)
    lv1 = torch.empty(A.n, dtype=torch.int32, device=dev)
    pa1 = torch.empty(A.n, dtype=torch.int32, device=dev)
    nl = torch.zeros(1, dtype=torch.int32, device=dev)
    same = True
    t_seq = 0.0
    for b in range(B):
        run = lambda: S.spmspv_bfs(Ap.handle, int(srcs[b]), lv1, pa1, nl, 0, stream)
        if b == 0:
            run()
        t_seq += _events_ms(run, stream, 1)
        same &= bool(torch.equal(lv1, lv[b * A.n:(b + 1) * A.n]) and torch.equal(pa1, pa[b * A.n:(b + 1) * A.n]))
    # the two forms side by side with the default schedule: every level as one
    # persistent launch over all sources, and 16 lanes
    forms = {}
    lv3 = torch.empty_like(lv)
    pa3 = torch.empty_like(pa)
    for name, ln in (("persistent", S.SPMSPV_LANES_PERSISTENT), ("lanes16", 16)):
        f = lambda: S.spmspv_msbfs(Ap.handle, B, ds, lv3, pa3, None, 0, ln, stream)
        f()
        forms[name + "_ms"] = _events_ms(f, stream, 2)
        forms[name + "_identical_results"] = bool(torch.equal(lv3, lv) and torch.equal(pa3, pa))
    del lv3, pa3
    out["msbfs"] = {"batched_ms": t_ms, "sequential_ms": t_seq, "speedup": t_seq / t_ms,
                    "tuned_lanes": tuned[0], "tuned_schedule": tuned[1],
                    "form": "persistent" if tuned[0] == 0 else "lanes", "identical_results": same}
    out["msbfs"].update(forms)
    params = selector_params()
    if params is not None:
        # the same searches with the learned schedule (push or pull per source
        # and level) inside the lanes, against the same sequential searches
        S.spmspv_selector_set(Ap.handle, params)
        lv2 = torch.empty_like(lv)
        pa2 = torch.empty_like(pa)
        msl = lambda: S.spmspv_msbfs(Ap.handle, B, ds, lv2, pa2, None, S.SPMSPV_SCHED_AUTO, 0, stream)
        msl()
        t_msl = _events_ms(msl, stream, 2)
        tuned = S.spmspv_last_tuned(Ap.handle)
        out["msbfs"].update({"learned_batched_ms": t_msl, "learned_speedup": t_seq / t_msl,
                             "learned_lanes": tuned[0],
                             "learned_identical_results": bool(torch.equal(lv2, lv) and torch.equal(pa2, pa))})
        del lv2, pa2
    del lv, pa

    # ACL from 256 seeds vs one seed at a time
    alpha, eps = 0.15, 1e-6
    p = torch.empty(B * A.n, dtype=torch.float32, device=dev)
    r = torch.empty(B * A.n, dtype=torch.float32, device=dev)
    acl = lambda: S.spmspv_acl(Ap.handle, B, ds, alpha, eps, 100000, p, r, None, 0, stream)
    acl()
    t_acl = _events_ms(acl, stream, 2)
    tuned = S.spmspv_last_tuned(Ap.handle)
    mass = float((p.view(B, -1).double().sum(1) + r.view(B, -1).double().sum(1) - 1).abs().max())
    p1 = torch.empty(A.n, dtype=torch.float32, device=dev)
    r1 = torch.empty(A.n, dtype=torch.float32, device=dev)
    t_seq = 0.0
    l1 = 0.0
    nseq = 32  # one seed at a time on a sample of the seeds, scaled to B
    for b in range(nseq):
        one = lambda: S.spmspv_acl(Ap.handle, 1, ds[b:b + 1], alpha, eps, 100000, p1, r1, None, 1, stream)
        if b == 0:
            one()
        t_seq += _events_ms(one, stream, 1)
        l1 = max(l1, float((p1 - p[b * A.n:(b + 1) * A.n]).abs().sum()))
    out["acl"] = {"alpha": alpha, "eps": eps, "batched_ms": t_acl,
                  "sequential_ms_scaled": t_seq * B / nseq, "sequential_sample": nseq,
                  "speedup": t_seq * B / nseq / t_acl, "tuned_lanes": tuned[0],
                  "tuned_schedule": tuned[1], "form": "persistent" if tuned[0] == 0 else "lanes",
                  "max_mass_error": mass, "max_l1_p_vs_single": l1}
    # the two forms side by side with the default schedule
    for name, ln in (("persistent", S.SPMSPV_LANES_PERSISTENT), ("lanes16", 16)):
        f = lambda: S.spmspv_acl(Ap.handle, B, ds, alpha, eps, 100000, p, r, None, ln, stream)
        f()
        out["acl"][name + "_ms"] = _events_ms(f, stream, 2)
    Ap.close()
    return out


def bench_selector_heldout(S, dev):
    """The learned selector on graphs it was not trained on (R-MAT s23 and the
    320^3 grid, BASELINE's held-out pair): per replayed BFS level, the regret
    t/t_best - 1 of the schedule it picks against the best of the 12 (and of
    the fixed default); per whole search (two sources each), the time of the
    fixed default, the learned schedule, the direction-optimizing rule and
    the best single fixed schedule (the autotuned fixed choice), levels and
    parents checked identical across all of them."""
    import torch
    import synth
    from paper_1610_07902_gb300 import selector
    params = selector_params()
    if params is None:
        return None
    out = {}
    for name, spec in selector.EVAL_GRAPHS:
        A = selector.make_graph(spec)
        Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC,
                         device=dev)
        srcs = synth.sources(A.colptr, 2, seed=7)
        r = selector.evaluate(Ad, A, srcs, params, reps=2, max_levels=24)
        lf = torch.empty(A.n, dtype=torch.int32, device=dev)
        pf = torch.empty_like(lf)
        nl = torch.zeros(1, dtype=torch.int32, device=dev)
        t_rule = 0.0
        same = True
        for src in srcs:
            S.spmspv_bfs(Ad.handle, int(src), lf, pf, nl, S.SPMSPV_SCHED_RULE)
            t_rule += _events_ms(lambda: S.spmspv_bfs(Ad.handle, int(src), lf, pf, nl, S.SPMSPV_SCHED_RULE),
                                 torch.cuda.current_stream(dev), 2)
            ts, ls, ps = selector.time_bfs(Ad, src, S.SPMSPV_SCHED_AUTO, 1)
            same &= bool(torch.equal(lf, ls) and torch.equal(pf, ps))
        tot = r["bfs_total_ms"]
        tot.update({"rule": t_rule, "auto_vs_rule": t_rule / tot["auto"],
                    "identical_results": bool(tot["identical_results"] and same)})
        tot.pop("per_schedule", None)
        out[name] = {"n": int(A.n), "nnz": int(A.nnz), "per_call_regret": r["per_call_regret"],
                     "bfs_total_ms": tot, "default_schedule": r["default_schedule"]}
        Ad.close()
        del A, lf, pf
        torch.cuda.empty_cache()
    return out


def profile_case(args, S, dev):
    """One kernel family on its own, for profiler captures: warm-up and
    timed steps of that workload only, one short JSON line.  Cases:
      pull     forced pull schedule (k_pull_scatter, k_pull_rows, k_pull_clear),
               (+,*) on R-MAT s<scale> with x of --nnz-x entries
      sortx    presort of x on the device (k_sortx_*) before the product
      bfs      BFS from one source under the fixed schedule (a graph loop)
      bfs_auto BFS under the learned schedule (persistent kernel + graph loop)
      grid_auto the same on the 3D grid of side --grid (persistent kernel)
      cc, mis, mcm   the graph algorithms (one graph loop each)
      msbfs    multi-source BFS from 64 sources (8 batched lanes)
      msbfs_persistent  the same, every level one persistent launch
      msbfs_learned  the same under the learned schedule (push launch + batched pull)
      batched  256 frontiers of log-uniform size in [1, 10^5] (R-MAT seed 4) as
               one persistent launch under schedule --sched
      batched_lanes  the same batch on 16 lanes
      auto     (+,*) product under the learned schedule (the selector runs in the
               work scan's last CTA), x of --nnz-x entries
      masked_min  (select2nd, min) product of x of --nnz-x entries (x(j) = j)
               under a complemented mask with half of the rows set"""
    import torch
    import synth
    stream = torch.cuda.current_stream(dev)
    case = args.case
    if case == "grid_auto":
        A = synth.grid3d(args.grid, args.grid, args.grid, 0.05, seed=3, values=False)
    elif case in ("batched", "batched_lanes"):
        A = synth.rmat(args.scale, EDGE_FACTOR, seed=4)
    else:
        A = synth.rmat(args.scale, EDGE_FACTOR, seed=SEED, values=case in ("pull", "sortx", "auto"))
    extra = {}
    sym = S.SPMSPV_CSC_SYMMETRIC if case in ("pull", "sortx", "batched", "batched_lanes") else \
        S.SPMSPV_CSC_PATTERN_SYMMETRIC
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val, flags=sym, device=dev)
    params = selector_params()
    if params is not None:
        S.spmspv_selector_set(Ad.handle, params)
    if case in ("auto", "masked_min"):
        xi_, xv_ = synth.frontier(A.n, min(args.nnz_x, A.n), seed=1, stream=2)
        xi = torch.from_numpy(xi_).to(dev)
        cap = A.m
        yi = torch.empty(cap, dtype=torch.int32, device=dev)
        nz = torch.zeros(1, dtype=torch.int32, device=dev)
        if case == "auto":
            xv = torch.from_numpy(xv_).to(dev)
            yv = torch.empty(cap, dtype=torch.float32, device=dev)
            step = lambda: S.spmspv_run(Ad.handle, S.SPMSPV_PLUS_TIMES_F32, xi, xv, xi_.size, None,
                                        S.SPMSPV_SCHED_AUTO, yi, yv, cap, nz, stream)
        else:
            rng = np.random.default_rng(3)
            bits = np.packbits((rng.random(A.m) < 0.5).astype(np.uint8), bitorder="little")
            bits = np.concatenate([bits, np.zeros((-len(bits)) % 4, np.uint8)]).view(np.int32)
            mask = torch.from_numpy(bits).to(dev)
            yv = torch.empty(cap, dtype=torch.int32, device=dev)
            step = lambda: S.spmspv_run(Ad.handle, S.SPMSPV_MIN_SELECT2ND_I32, xi, xi, xi_.size, mask,
                                        S.SPMSPV_MASK_COMPLEMENT, yi, yv, cap, nz, stream)
    elif case in ("pull", "sortx"):
        xi_, xv_ = synth.frontier(A.n, min(args.nnz_x, A.n), seed=1, stream=2)
        xi, xv = torch.from_numpy(xi_).to(dev), torch.from_numpy(xv_).to(dev)
        cap = A.m
        yi = torch.empty(cap, dtype=torch.int32, device=dev)
        yv = torch.empty(cap, dtype=torch.float32, device=dev)
        nz = torch.zeros(1, dtype=torch.int32, device=dev)
        opts = S.SPMSPV_SCHED_OPT(11) if case == "pull" else S.SPMSPV_SORT_X
        step = lambda: S.spmspv_run(Ad.handle, S.SPMSPV_PLUS_TIMES_F32, xi, xv, xi_.size, None, opts, yi, yv,
                                    cap, nz, stream)
    elif case in ("bfs", "bfs_auto", "grid_auto"):
        src = int(synth.sources(A.colptr, 1, seed=2)[0]) if case != "grid_auto" else \
            (args.grid // 2) * args.grid * args.grid + (args.grid // 2) * args.grid + args.grid // 2
        lv = torch.empty(A.n, dtype=torch.int32, device=dev)
        pa = torch.empty_like(lv)
        nl = torch.zeros(1, dtype=torch.int32, device=dev)
        opts = S.SPMSPV_SCHED_OPT(5) if case == "bfs" else S.SPMSPV_SCHED_AUTO
        step = lambda: S.spmspv_bfs(Ad.handle, src, lv, pa, nl, opts, stream)
    elif case == "cc":
        lab = torch.empty(A.n, dtype=torch.int32, device=dev)
        step = lambda: S.spmspv_cc(Ad.handle, lab, None, 0, stream)
    elif case == "mis":
        g = torch.Generator(device="cpu").manual_seed(7)
        prio = torch.randperm(A.n, generator=g).to(torch.int32).to(dev)
        ins = torch.empty(A.n, dtype=torch.int32, device=dev)
        step = lambda: S.spmspv_mis(Ad.handle, prio, ins, None, 0, stream)
    elif case == "mcm":
        mr = torch.empty(A.m, dtype=torch.int32, device=dev)
        mc = torch.empty(A.n, dtype=torch.int32, device=dev)
        step = lambda: S.spmspv_mcm(Ad.handle, mr, mc, None, None, 0, stream)
    elif case in ("batched", "batched_lanes"):
        B = 256
        rng = np.random.default_rng(4)
        sizes = np.maximum(1, np.floor(10 ** rng.uniform(0, 5, B))).astype(np.int64)
        fronts = [synth.frontier(A.n, int(min(f, A.n)), seed=100 + b, stream=2) for b, f in enumerate(sizes)]
        x_cnt = np.array([f[0].shape[0] for f in fronts], np.int32)
        x_off = np.concatenate([[0], np.cumsum(x_cnt)[:-1]]).astype(np.int32)
        td = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        bx = (td(x_off), td(x_cnt), td(np.concatenate([f[0] for f in fronts])),
              td(np.concatenate([f[1] for f in fronts])))
        by = (td((np.arange(B, dtype=np.int64) * A.m).astype(np.int32)), td(np.full(B, A.m, np.int32)))
        yi = torch.empty(B * A.m, dtype=torch.int32, device=dev)
        yv = torch.empty(B * A.m, dtype=torch.float32, device=dev)
        nz = torch.zeros(B, dtype=torch.int32, device=dev)
        lanes = S.SPMSPV_LANES_PERSISTENT if case == "batched" else 16
        extra["products"] = int(sum(int(np.diff(A.colptr)[f[0]].sum()) for f in fronts))
        step = lambda: S.spmspv_run_batched(Ad.handle, S.SPMSPV_PLUS_TIMES_F32, B, *bx, None, 0,
                                            S.SPMSPV_SCHED_OPT(args.sched), *by, yi, yv, nz, lanes, stream)
    elif case in ("msbfs", "msbfs_persistent", "msbfs_learned"):
        B = 64
        srcs = torch.from_numpy(synth.sources(A.colptr, B, seed=5).astype(np.int32)).to(dev)
        lv = torch.empty(B * A.n, dtype=torch.int32, device=dev)
        pa = torch.empty_like(lv)
        lanes = 8 if case == "msbfs" else S.SPMSPV_LANES_PERSISTENT
        opts = S.SPMSPV_SCHED_AUTO if case == "msbfs_learned" else S.SPMSPV_SCHED_OPT(args.sched)
        step = lambda: S.spmspv_msbfs(Ad.handle, B, srcs, lv, pa, None, opts, lanes, stream)
    else:
        raise SystemExit("unknown case %s" % case)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    t = _events_ms(lambda: [step() for _ in range(args.steps)], stream, 1) / max(args.steps, 1)
    if "products" in extra:
        extra["gteps"] = extra["products"] / (t * 1e-3) / 1e9
    if case == "batched":
        ph, waves = S.spmspv_batched_phase_times(Ad.handle)
        extra["phases_ms"] = dict(zip(["scan", "plan", "tile_starts", "expand", "merge", "launch",
                                       "direct_expand", "direct_compact"], [round(float(v), 4) for v in ph]))
        extra["waves"] = waves
    print(json.dumps(dict({"case": case, "scale": args.scale, "ms_per_step": t,
                           "status": S.spmspv_device_status(Ad.handle)}, **extra)), flush=True)
    Ad.close()


def reference_arm(args, rank):
    if rank != 0:
        return
    import synth
    A = synth.rmat(SCALE, EDGE_FACTOR, seed=SEED)
    x_idx, x_val = synth.frontier(A.n, F, seed=1, stream=2)
    import oracle
    # each step: the oracle on a 10^4-entry slice of x (a bounded sample of the workload)
    fs = 10_000
    for i in range(args.warmup):
        sl = slice((i * fs) % F, (i * fs) % F + fs)
        oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, oracle.PLUS_TIMES, x_idx[sl], x_val[sl],
                      with_absum=False)
    W, t = 0, 0.0
    for i in range(args.steps):
        sl = slice((i * fs) % F, (i * fs) % F + fs)
        t0 = time.perf_counter()
        r = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, oracle.PLUS_TIMES, x_idx[sl], x_val[sl],
                          with_absum=False)
        t += time.perf_counter() - t0
        W += r.nmult
    v = W / t / 1e9
    line = {"metric": METRIC, "value": v, "unit": "GTEPS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": "x slices of %d entries" % fs},
            "cpu_baseline": {"value": v, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                             "sample": "%d steps of a %d-entry slice of x" % (args.steps, fs)},
            "e2e": {"value": v, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--scale", type=int, default=SCALE,
                    help="R-MAT scale (smaller only for profiler captures)")
    ap.add_argument("--nnz-x", type=int, default=F)
    ap.add_argument("--buckets-only", action="store_true",
                    help="run the headline product in the bucketed form even where the direct form applies")
    ap.add_argument("--kernels-only", action="store_true",
                    help="warm-up and timed steps only (for profiler captures)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the BFS (fixed vs learned) and batched measurements")
    ap.add_argument("--case", default=None,
                    choices=["pull", "sortx", "bfs", "bfs_auto", "grid_auto", "cc", "mis", "mcm", "msbfs", "msbfs_persistent",
                             "msbfs_learned", "batched",
                             "batched_lanes", "auto", "masked_min"],
                    help="run one kernel family only (for profiler captures)")
    ap.add_argument("--grid", type=int, default=64, help="grid side of --case grid_auto")
    ap.add_argument("--sched", type=int, default=5, help="push schedule of --case batched / msbfs")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        reference_arm(args, rank)
        return

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_1610_07902_gb300 import spmspv as S
    S.load()
    if args.case:
        profile_case(args, S, torch.device("cuda", local))
        return

    F_ = args.nnz_x
    A, x_idx, x_val = make_inputs(args.scale, F_)
    workload = WORKLOAD if (args.scale, F_) == (SCALE, F) else "rmat%d_ef16_f%d_plus_times_f32" % (
        args.scale, F_)
    dev = torch.device("cuda", local)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val, device=dev)
    xi = torch.from_numpy(x_idx).to(dev)
    xv = torch.from_numpy(x_val).to(dev)
    cap = min(A.m, A.nnz)
    y_idx = torch.empty(cap, dtype=torch.int32, device=dev)
    y_val = torch.empty(cap, dtype=torch.float32, device=dev)
    nnz_y = torch.zeros(1, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    opts = S.SPMSPV_SORTED_OUT | (S.SPMSPV_BUCKETS_ONLY if args.buckets_only else 0)

    def step():
        S.spmspv_run(Ad.handle, S.SPMSPV_PLUS_TIMES_F32, xi, xv, F_, None, opts, y_idx, y_val, cap,
                     nnz_y, stream)

    sampler = ClockSampler(local)
    time.sleep(0.3)
    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    W = S.spmspv_last_work(Ad.handle)
    ny = int(nnz_y.item())
    assert S.spmspv_device_status(Ad.handle) == 0

    # timed region: K steps, L2 flushed before each, device time by CUDA events
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms_median = float(np.median(step_ms))
    t_ms = sum(step_ms)
    t_ms, gteps = replica_summary(t_ms, W, args.steps, world, dev)
    ms_per_step = t_ms / args.steps
    if args.kernels_only:
        sampler.stop()
        if rank == 0:
            print(json.dumps({"workload": workload, "ms_per_step": ms_per_step, "value": gteps,
                              "unit": "GTEPS", "kernels_only": True}), flush=True)
        Ad.close()
        return

    # per-stage device time (events around every kernel, separate pass)
    S.spmspv_profile_begin(Ad.handle)
    nprof = max(20, min(args.steps, 200))
    for _ in range(nprof):
        flush.zero_()
        step()
    stage_ms, ncalls = S.spmspv_profile_end(Ad.handle)
    stage_avg = [s / ncalls for s in stage_ms]

    # end to end through the C ABI from pinned host memory: copy x in, run, copy y out
    hx_i = torch.from_numpy(x_idx).pin_memory()
    hx_v = torch.from_numpy(x_val).pin_memory()
    hy_i = torch.empty(cap, dtype=torch.int32).pin_memory()
    hy_v = torch.empty(cap, dtype=torch.float32).pin_memory()
    ne2 = max(10, min(args.steps, 100))
    e2e_ms = 0.0
    k = 0
    for i in range(ne2 + 2):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # one call of the C ABI with host buffers: x in, the product, nnz(y)
        # read first (one synchronisation), then that many entries of y out
        k = S.spmspv_run_host(Ad.handle, S.SPMSPV_PLUS_TIMES_F32, hx_i, hx_v, F_, None, opts, hy_i, hy_v, cap,
                              stream)
        if i >= 2:
            e2e_ms += (time.perf_counter() - t0) * 1e3
    assert k == ny
    e2e_gteps = W * ne2 * world / (e2e_ms * 1e-3) / 1e9 if world == 1 else None
    clocks = sampler.stop()

    peak, peak_kind = load_peaks()
    form = product_form(A.m, W, args.buckets_only)
    names, kname, per_unit, traffic_src, units, alg, dom, achieved = stage_roofline(S, form, F_, W, ny,
                                                                                    stage_avg)
    path_bytes = compulsory_bytes(F_, W, ny)
    path_gbs = path_bytes / (ms_per_step * 1e-3) / 1e9

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, calls, tt = time_oracle(A, x_idx, x_val)
        nproc, model = host_cpu()
        cpu = {"value": v, "unit": "GTEPS", "cores": 1, "kind": "oracle",
               "sample": "%d full calls of the workload (%.1f s)" % (calls, tt),
               "median_ms_per_call": 1e3 * time_oracle.median_s, "host_threads": nproc,
               "host_cpu": model}

    extras = {}
    if rank == 0 and not args.no_extras:
        import synth
        if form == "direct":
            extras["bucketed_form"] = bench_bucketed_form(S, Ad, xi, xv, F_, y_idx, y_val, cap, nnz_y, stream,
                                                          flush, peak)
        # the same graph at the smaller frontiers of the sweep (host-launched calls)
        sweep = {}
        for fs in (100, 10_000):
            sxi, sxv = synth.frontier(A.n, fs, seed=1, stream=2)
            dxi, dxv = torch.from_numpy(sxi).to(dev), torch.from_numpy(sxv).to(dev)
            run = lambda: S.spmspv_run(Ad.handle, S.SPMSPV_PLUS_TIMES_F32, dxi, dxv, fs, None, opts,
                                       y_idx, y_val, cap, nnz_y, stream)
            for _ in range(5):
                run()
            reps = 200
            tms = _events_ms(lambda: [run() for _ in range(reps)], stream, 1) / reps
            ws_ = S.spmspv_last_work(Ad.handle)
            cb = compulsory_bytes(fs, ws_, int(nnz_y.item()))
            tg = graph_us_per_call(lambda cs: S.spmspv_run(Ad.handle, S.SPMSPV_PLUS_TIMES_F32, dxi, dxv, fs,
                                                            None, opts, y_idx, y_val, cap, nnz_y, cs), stream)
            sweep["nnz_x_%d" % fs] = {"us_per_call": 1e3 * tms, "graph_us_per_call": tg, "products": ws_,
                                       "gteps": ws_ / (tms * 1e-3) / 1e9, "compulsory_bytes": cb,
                                       "path_frac": cb / (tms * 1e-3) / 1e9 / peak}
        sweep["note"] = ("back-to-back host-launched calls, L2 not flushed between them; "
                         "graph_us_per_call: 100 calls captured in one CUDA graph and replayed")
        extras["sweep_rmat"] = sweep
        extras["er_spmspv"] = bench_er(S, dev, stream)
        extras["sorted_x_rmat"] = bench_sorted_x(S, A, Ad, dev, stream, flush, y_idx, y_val, cap, nnz_y)
        params = selector_params()
        extras["bfs_rmat"] = bench_bfs(S, A, dev, stream, "rmat s%d ef16 seed 1" % args.scale,
                                       synth.sources(A.colptr, 64, seed=2), params)
        extras["cc_rmat"] = bench_cc(S, A, dev, stream)
        extras["mis_rmat"] = bench_mis(S, A, dev, stream)
        extras["matching_rmat"] = bench_mcm(S, A, dev, stream)
        del Ad
        G = synth.grid3d(256, 256, 256, 0.05, seed=3)
        extras["bfs_grid"] = bench_bfs(S, G, dev, stream, "grid 256^3 7-point, 5% edges removed",
                                       [128 * 65536 + 128 * 256 + 128], params, pt_frontiers=True)
        del G
        extras["batched"] = bench_batched(S, dev, stream)
        extras["dcsc_hypersparse"] = bench_dcsc(S, dev, stream, flush)
        extras["selector_weights"] = "trained" if params is not None else "absent (AUTO not run)"
        extras["selector_heldout"] = bench_selector_heldout(S, dev)

    line = {
        "metric": METRIC, "value": gteps, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "ms_median": ms_median,
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload, "graph": "rmat s%d ef16 symmetrised seed 1" % args.scale,
                   "m": A.m, "nnz": A.nnz, "nnz_x": F_, "products": W, "nnz_y": ny, "form": form,
                   "semiring": "plus_times_f32", "l2": "flushed (256 MiB write) before each step",
                   "parallelism": "replicas" if world > 1 else "single_gpu"},
        "roofline": {"bound": "hbm", "kernel": kname, "stage": names[dom], "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak,
                     "traffic": per_unit * units[dom] if per_unit else None,
                     "traffic_unit": "bytes per launch",
                     "traffic_source": ("%s (ncu capture of these kernel sources, %s, scaled by the "
                                        "launch's units)" % (traffic_src, kernels_hash())
                                        if per_unit else "no capture of the current kernel sources"),
                     "peak_kind": peak_kind, "alg_bytes_per_launch": alg[dom],
                     "avg_launch_ms": stage_avg[dom], "frac_nominal": achieved / NOMINAL_HBM_GBS},
        "path_roofline": {"compulsory_bytes": path_bytes, "achieved": path_gbs, "peak": peak,
                          "unit": "GB/s", "frac": path_gbs / peak, "peak_kind": peak_kind,
                          "frac_nominal": path_gbs / NOMINAL_HBM_GBS},
        "stages_ms": {names[s]: stage_avg[s] for s in names},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_gteps, "unit": "GTEPS", "h2d_bytes_per_step": 8 * F_,
                "d2h_bytes_per_step": 4 + 8 * ny,
                "note": ("spmspv_run_host with pinned host x and y: x in, the product, nnz(y) read "
                         "(one synchronisation), then y out; host wall clock per call")},
        "gpu_launches": 3 * args.steps,
        "clocks": clocks,
    }
    line.update(extras)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if not extras:
        Ad.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
