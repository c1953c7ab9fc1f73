"""The row-split form's product on a GPU (one NCCL rank): the rank's row
block through the library (the default local product), against the oracle
restricted to the same rows."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth
from gpu_util import SEMIRING_TO_ORACLE, compare, need_gpu, x_values

pytestmark = pytest.mark.gpu


def test_row_block_product_on_the_gpu():
    torch = need_gpu()
    import torch.distributed as dist
    from paper_1610_07902_gb300 import rowsplit
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        A = synth.rmat(14, seed=12)
        r0 = A.m // 3
        rs = rowsplit.RowSplitSpMSpV(A.m, A.n, A.colptr, A.rowidx, A.val, bounds=[r0, A.m])
        xi, xf = synth.frontier(A.n, 2000, seed=4)
        keep = np.zeros(A.m, np.uint8)
        keep[r0:] = 1
        for sem in (0, 1, 2):
            xv = x_values(sem, xi, xf)
            yi, yv = rs.multiply(sem, torch.from_numpy(xi).cuda(), None if xv is None else torch.from_numpy(xv).cuda())
            # rows below r0 are not this rank's: the oracle with them masked out
            ref = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, SEMIRING_TO_ORACLE[sem], xi, xv, 1 - keep, True)
            compare(sem, ref, yi.cpu().numpy(), None if yv is None else yv.cpu().numpy())
        rs.close()
    finally:
        dist.destroy_process_group()
