"""Row-split SpMSpV over several GPUs, one process per GPU.

Each rank holds the row block A(r0:r1, :) in CSC on its own GPU and the
entries of x it produced; a product is one allgather of x (every rank needs
all of it: the O(t f) access to x that Sec. II-F charges to the row-split
scheme), then the local product y(r0:r1) = A(r0:r1, :) x on the rank's GPU
through the C ABI, with no synchronisation on y (each rank owns its rows;
Sec. II-F).  y stays distributed: rank g returns the entries of rows
[r0, r1), with global row ids, in ascending order, so the ranks' outputs
concatenated in rank order are the single-GPU y.

Row blocks are cut at equal shares of the stored entries (R-MAT rows are
skewed, so equal row counts would not balance the products).

The exchange uses torch.distributed (NCCL between GPUs; the tests run the
same code on gloo ranks on the CPU, with the local product passed in).
"""
from __future__ import annotations

import numpy as np


def row_bounds(m, rowidx, world):
    """Row block boundaries b[0] = 0 <= b[1] <= ... <= b[world] = m that give
    every block about nnz/world stored entries (host arrays)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    deg = np.bincount(np.asarray(rowidx, dtype=np.int64), minlength=m)[:m]
    cum = np.concatenate([[0], np.cumsum(deg)])
    total = int(cum[-1])
    b = [0]
    for g in range(1, world):
        target = total * g // world
        r = int(np.searchsorted(cum, target, side="left"))
        b.append(min(max(r, b[-1]), m))
    b.append(m)
    return np.asarray(b, dtype=np.int64)


def split_rows(colptr, rowidx, val, r0, r1):
    """The row block A(r0:r1, :) as a CSC with r1 - r0 rows (row ids rebased
    to r0) and the same n columns; row order inside each column is kept."""
    colptr = np.asarray(colptr, dtype=np.int64)
    rowidx = np.asarray(rowidx, dtype=np.int32)
    keep = (rowidx >= r0) & (rowidx < r1)
    n = colptr.shape[0] - 1
    col_of = np.repeat(np.arange(n, dtype=np.int64), np.diff(colptr))
    cnt = np.bincount(col_of[keep], minlength=n)
    lcp = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int32)
    lri = (rowidx[keep] - r0).astype(np.int32)
    lva = None if val is None else np.asarray(val, dtype=np.float32)[keep]
    return lcp, lri, lva


def allgather_x(x_idx, x_val, group=None):
    """Every rank's x entries, concatenated in rank order, on every rank.
    x_idx int32 and x_val (float32/int32, or None for a pattern semiring) are
    tensors on the rank's device; sizes may differ between ranks (and be 0)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    dev = x_idx.device
    n_local = torch.tensor([x_idx.numel()], dtype=torch.int64, device=dev)
    sizes = [torch.zeros_like(n_local) for _ in range(world)]
    dist.all_gather(sizes, n_local, group=group)
    sizes = [int(s.item()) for s in sizes]
    cap = max(max(sizes), 1)

    def gather(t, fill):
        buf = torch.full((cap,), fill, dtype=t.dtype, device=dev)
        buf[:t.numel()] = t
        parts = [torch.empty_like(buf) for _ in range(world)]
        dist.all_gather(parts, buf, group=group)
        return torch.cat([p[:s] for p, s in zip(parts, sizes)])

    xi = gather(x_idx.to(torch.int32), -1)
    xv = None if x_val is None else gather(x_val, 0)
    return xi, xv


class RowSplitSpMSpV:
    """One rank's part of a row-split matrix.

    A: the whole matrix as host CSC arrays (m, n, colptr, rowidx, val) - each
    rank keeps only its row block.  local_multiply(semiring, x_idx, x_val) ->
    (y_idx, y_val) computes the product of the local block with the gathered
    x; by default it is the library's spmspv_run on the rank's GPU (a
    CscMatrix of the block), with no fallback when no GPU is there.
    """

    def __init__(self, m, n, colptr, rowidx, val=None, group=None, device=None, local_multiply=None,
                 bounds=None):
        import torch.distributed as dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.m, self.n = int(m), int(n)
        self.bounds = row_bounds(self.m, rowidx, self.world) if bounds is None else np.asarray(bounds)
        self.r0, self.r1 = int(self.bounds[self.rank]), int(self.bounds[self.rank + 1])
        self.colptr, self.rowidx, self.val = split_rows(colptr, rowidx, val, self.r0, self.r1)
        self._Ad = None
        if local_multiply is None:
            from . import spmspv as S
            self._Ad = S.CscMatrix(self.r1 - self.r0, self.n, self.colptr, self.rowidx, self.val,
                                   device=device or "cuda")
            Ad = self._Ad

            def local_multiply(semiring, xi, xv):
                yi, yv, _ = Ad.multiply(semiring, xi, xv)
                return yi, yv
        self.local_multiply = local_multiply

    def multiply(self, semiring, x_idx, x_val):
        """y(r0:r1) for this rank's x entries (the whole x is their union over
        the ranks; an index must not appear on two ranks)."""
        xi, xv = allgather_x(x_idx, x_val, self.group)
        yi, yv = self.local_multiply(semiring, xi, xv)
        return yi + self.r0, yv

    def close(self):
        if self._Ad is not None:
            self._Ad.close()
            self._Ad = None
