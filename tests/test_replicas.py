"""The N > 1 path of bench.py (replicas only): two gloo ranks on the CPU take
the slowest rank's time and report the products of both ranks over it."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_ms = 10.0 if rank == 0 else 25.0  # rank 1 is the slower one
    out[rank] = bench.replica_summary(t_ms, 1_000_000, 4, world, "cpu")
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        t_ms, gteps = res[rank]
        assert t_ms == 25.0
        assert gteps == pytest.approx(1_000_000 * 4 * 2 / 25e-3 / 1e9)


def test_one_rank_needs_no_group():
    import bench
    t_ms, gteps = bench.replica_summary(8.0, 500, 2, 1, "cpu")
    assert t_ms == 8.0 and gteps == pytest.approx(500 * 2 / 8e-3 / 1e9)
