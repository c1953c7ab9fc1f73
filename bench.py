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
    while t_total < budget_s or calls == 0:
        t0 = time.perf_counter()
        r = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, oracle.PLUS_TIMES, x_idx, x_val,
                          with_absum=False)
        t_total += time.perf_counter() - t0
        W_total += r.nmult
        calls += 1
        if calls >= 20:
            break
    return W_total / t_total / 1e9, calls, t_total


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
    ap.add_argument("--kernels-only", action="store_true",
                    help="warm-up and timed steps only (for profiler captures)")
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
    opts = S.SPMSPV_SORTED_OUT

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
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    if world > 1:
        dist.barrier()
        tt = torch.tensor([t_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms = float(tt.item())
    ms_per_step = t_ms / args.steps
    gteps = W * args.steps * world / (t_ms * 1e-3) / 1e9
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
    hn = torch.zeros(1, dtype=torch.int32).pin_memory()
    xi2 = torch.empty_like(xi)
    xv2 = torch.empty_like(xv)
    ne2 = max(10, min(args.steps, 100))
    e2e_ms = 0.0
    for i in range(ne2 + 2):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xi2.copy_(hx_i, non_blocking=True)
        xv2.copy_(hx_v, non_blocking=True)
        S.spmspv_run(Ad.handle, S.SPMSPV_PLUS_TIMES_F32, xi2, xv2, F_, None, opts, y_idx, y_val,
                     cap, nnz_y, stream)
        hn.copy_(nnz_y, non_blocking=True)
        hy_i[:ny].copy_(y_idx[:ny], non_blocking=True)
        hy_v[:ny].copy_(y_val[:ny], non_blocking=True)
        torch.cuda.synchronize()
        if i >= 2:
            e2e_ms += (time.perf_counter() - t0) * 1e3
    assert int(hn.item()) == ny
    e2e_gteps = W * ne2 * world / (e2e_ms * 1e-3) / 1e9 if world == 1 else None
    clocks = sampler.stop()

    peak, peak_kind = load_peaks()
    names = {S.SPMSPV_STAGE_SCAN: "work_scan", S.SPMSPV_STAGE_SCATTER: "expand_scatter",
             S.SPMSPV_STAGE_MERGE: "bucket_merge"}
    alg = {S.SPMSPV_STAGE_SCAN: 16 * F_, S.SPMSPV_STAGE_SCATTER: 8 * W,
           S.SPMSPV_STAGE_MERGE: 8 * ny}
    dom = max(names, key=lambda s: stage_avg[s])
    achieved = alg[dom] / (stage_avg[dom] * 1e-3) / 1e9
    path_bytes = compulsory_bytes(F_, W, ny)
    path_gbs = path_bytes / (ms_per_step * 1e-3) / 1e9

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, calls, tt = time_oracle(A, x_idx, x_val)
        cpu = {"value": v, "unit": "GTEPS", "cores": 1, "kind": "oracle",
               "sample": "%d full calls of the workload (%.1f s)" % (calls, tt)}

    line = {
        "metric": METRIC, "value": gteps, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload, "graph": "rmat s%d ef16 symmetrised seed 1" % args.scale,
                   "m": A.m, "nnz": A.nnz, "nnz_x": F_, "products": W, "nnz_y": ny,
                   "semiring": "plus_times_f32", "l2": "flushed (256 MiB write) before each step",
                   "parallelism": "replicas" if world > 1 else "single_gpu"},
        "roofline": {"bound": "hbm", "kernel": names[dom], "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "peak_kind": peak_kind, "alg_bytes_per_launch": alg[dom],
                     "avg_launch_ms": stage_avg[dom]},
        "path_roofline": {"compulsory_bytes": path_bytes, "achieved": path_gbs, "peak": peak,
                          "unit": "GB/s", "frac": path_gbs / peak, "peak_kind": peak_kind},
        "stages_ms": {names[s]: stage_avg[s] for s in names},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_gteps, "unit": "GTEPS", "h2d_bytes_per_step": 8 * F_,
                "d2h_bytes_per_step": 4 + 8 * ny},
        "gpu_launches": 3 * args.steps,
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    Ad.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
