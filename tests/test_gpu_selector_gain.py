"""What the trained selector gains over the method without it.

The committed network (paper_1610_07902_gb300/selector_weights.json, trained
on the GPU by the library's own kernels on timings of R-MAT scales 16-21 and
2D/3D grids) picks a schedule per BFS level.  On a scale-free graph the plain
fixed schedule pushes every level, while the network pulls the dense middle
levels.  The test runs whole BFS (one graph launch each) from several sources
under both, requires identical levels and parents, and requires the learned
schedule to be faster in total.  The measured ratio is printed.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _bfs_ms(torch, S, Ad, src, opts, level, parent, nl, reps=3):
    run = lambda: S.spmspv_bfs(Ad.handle, int(src), level, parent, nl, opts)
    run()
    best = float("inf")
    st = torch.cuda.current_stream()
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        run()
        b.record(st)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def test_learned_schedule_beats_fixed_on_rmat_bfs():
    torch = need_gpu()
    from paper_1610_07902_gb300 import selector, spmspv as S
    S.load()
    params, meta = selector.load()
    assert meta.get("samples", 0) > 0
    A = synth.rmat(20, seed=31, values=False)  # not one of the training graphs
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, None, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
    S.spmspv_selector_set(Ad.handle, params)
    fixed = S.SPMSPV_SCHED_OPT(S.spmspv_default_schedule(Ad.handle))
    dev = Ad.colptr.device
    lf = torch.empty(A.n, dtype=torch.int32, device=dev)
    pf = torch.empty(A.n, dtype=torch.int32, device=dev)
    la = torch.empty_like(lf)
    pa = torch.empty_like(pf)
    nl = torch.zeros(1, dtype=torch.int32, device=dev)
    t_fixed = t_auto = 0.0
    srcs = synth.sources(A.colptr, 6, seed=13)
    for src in srcs:
        t_fixed += _bfs_ms(torch, S, Ad, src, fixed, lf, pf, nl)
        t_auto += _bfs_ms(torch, S, Ad, src, S.SPMSPV_SCHED_AUTO, la, pa, nl)
        assert torch.equal(lf, la) and torch.equal(pf, pa)
    lv, par, _, _, _ = oracle.bfs(A.colptr, A.rowidx, int(srcs[0]))
    _bfs_ms(torch, S, Ad, srcs[0], S.SPMSPV_SCHED_AUTO, la, pa, nl, reps=1)
    np.testing.assert_array_equal(la.cpu().numpy(), lv)
    np.testing.assert_array_equal(pa.cpu().numpy(), par)
    print("rmat20 BFS x%d: fixed %.2f ms, learned %.2f ms, speedup %.2fx"
          % (len(srcs), t_fixed, t_auto, t_fixed / t_auto))
    assert t_auto < t_fixed
    Ad.close()
