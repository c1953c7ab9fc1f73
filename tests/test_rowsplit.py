"""The row-split multi-GPU form (paper_1610_07902_gb300.rowsplit) on gloo
ranks on the CPU: row blocks, the allgather of x, and that the ranks' y
pieces concatenated in rank order are the product of the whole matrix.  The
local product of each block is the oracle here (no GPU in these tests); on
GPUs it is the library's spmspv_run."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import synth
from gpu_util import SEMIRING_TO_ORACLE, x_values


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_row_bounds_balance_entries():
    from paper_1610_07902_gb300 import rowsplit
    A = synth.rmat(12, seed=3)
    deg = np.bincount(A.rowidx, minlength=A.m)
    for world in (1, 2, 3, 8):
        b = rowsplit.row_bounds(A.m, A.rowidx, world)
        assert b[0] == 0 and b[-1] == A.m and np.all(np.diff(b) >= 0)
        per = [int(deg[b[g]:b[g + 1]].sum()) for g in range(world)]
        assert sum(per) == A.nnz
        assert max(per) - A.nnz / world <= deg.max() + 1


def test_split_rows_blocks_make_the_product():
    from paper_1610_07902_gb300 import rowsplit
    A = synth.rmat(11, seed=5)
    xi, xf = synth.frontier(A.n, 300, seed=2)
    for sem in (0, 1, 2):
        xv = x_values(sem, xi, xf)
        full = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, SEMIRING_TO_ORACLE[sem], xi, xv)
        b = rowsplit.row_bounds(A.m, A.rowidx, 3)
        idx, val = [], []
        for g in range(3):
            cp, ri, va = rowsplit.split_rows(A.colptr, A.rowidx, A.val, int(b[g]), int(b[g + 1]))
            assert np.all(np.diff(cp) >= 0) and (ri.size == 0 or (ri.min() >= 0 and ri.max() < b[g + 1] - b[g]))
            part = oracle.spmspv(int(b[g + 1] - b[g]), cp, ri, va, SEMIRING_TO_ORACLE[sem], xi, xv)
            idx.append(part.idx + b[g])
            val.append(part.val)
        np.testing.assert_array_equal(np.concatenate(idx), full.idx)
        if sem != 2:
            np.testing.assert_array_equal(np.concatenate(val), full.val)


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1610_07902_gb300 import rowsplit
    A = synth.rmat(11, seed=7)

    def local(sem, xi_t, xv_t):
        # the local product of this rank's block: the oracle (the CPU stands in for the GPU)
        r = oracle.spmspv(rs.r1 - rs.r0, rs.colptr, rs.rowidx, rs.val, SEMIRING_TO_ORACLE[sem],
                          xi_t.numpy(), None if xv_t is None else xv_t.numpy())
        yv = None if sem == 2 else torch.from_numpy(np.asarray(r.val, np.float64))
        return torch.from_numpy(r.idx.astype(np.int32)), yv

    rs = rowsplit.RowSplitSpMSpV(A.m, A.n, A.colptr, A.rowidx, A.val, local_multiply=local)
    xi, xf = synth.frontier(A.n, 500, seed=9)
    res = {}
    for sem in (0, 1, 2):
        xv = x_values(sem, xi, xf)
        mine = (xi % world) == rank   # this rank's share of x (the last rank drops some)
        if rank == world - 1:
            mine = mine & (xi % 3 != 0)
        xi_t = torch.from_numpy(xi[mine].astype(np.int32))
        xv_t = None if xv is None else torch.from_numpy(xv[mine])
        yi, yv = rs.multiply(sem, xi_t, xv_t)
        res[sem] = (yi.numpy(), None if yv is None else yv.numpy())
        # the gathered x is every rank's share, in rank order
        gi, _ = rowsplit.allgather_x(xi_t, xv_t)
        res["x%d" % sem] = gi.numpy()
    out[rank] = (rs.r0, rs.r1, res)
    # ranks without any x entry (only rank 1 has five)
    empty = torch.zeros(0, dtype=torch.int32)
    yi, _ = rs.multiply(2, torch.from_numpy(xi[:5].astype(np.int32)) if rank == 1 else empty, None)
    out["empty%d" % rank] = yi.numpy()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_assemble_the_product(world):
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    A = synth.rmat(11, seed=7)
    xi, xf = synth.frontier(A.n, 500, seed=9)
    bounds = [res[g][:2] for g in range(world)]
    assert bounds[0][0] == 0 and bounds[-1][1] == A.m
    assert all(bounds[g][1] == bounds[g + 1][0] for g in range(world - 1))
    for sem in (0, 1, 2):
        xv = x_values(sem, xi, xf)
        shares = []
        for g in range(world):
            mine = (xi % world) == g
            if g == world - 1:
                mine = mine & (xi % 3 != 0)
            shares.append(np.nonzero(mine)[0])
        used = np.concatenate(shares)
        full = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, SEMIRING_TO_ORACLE[sem], xi[used],
                             None if xv is None else xv[used])
        for g in range(world):
            np.testing.assert_array_equal(res[g][2]["x%d" % sem], xi[used])
        yi = np.concatenate([res[g][2][sem][0] for g in range(world)])
        np.testing.assert_array_equal(yi, full.idx)
        if sem != 2:
            yv = np.concatenate([res[g][2][sem][1] for g in range(world)])
            np.testing.assert_allclose(yv, full.val, rtol=1e-12, atol=0)
    ref = oracle.spmspv(A.m, A.colptr, A.rowidx, None, oracle.OR_AND, xi[:5] if world > 1 else xi[:0], None)
    got = np.concatenate([res["empty%d" % g] for g in range(world)])
    np.testing.assert_array_equal(got, ref.idx)
