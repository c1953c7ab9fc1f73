"""Helpers shared by the GPU parity tests (host-side marshalling only)."""
import numpy as np
import pytest

import oracle

SEMIRING_TO_ORACLE = {0: oracle.PLUS_TIMES, 1: oracle.MIN_SELECT2ND, 2: oracle.OR_AND}
FP_TOL = 1e-5  # |y_gpu - y_fp64| <= FP_TOL * sum_j |A(i,j) x(j)|


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def mask_bits(mask_u8):
    """uint8[m] (1 = in the mask) -> uint32 bitmap words (bit i%32 of word i/32)."""
    m = mask_u8.shape[0]
    words = (m + 31) // 32
    padded = np.zeros(words * 32, np.uint8)
    padded[:m] = mask_u8 != 0
    bits = np.packbits(padded, bitorder="little")
    return bits.view("<u4").astype(np.uint32) if bits.size else np.zeros(0, np.uint32)


def x_values(semiring, x_idx, x_val_f32):
    if semiring == 0:
        return x_val_f32.astype(np.float32)
    if semiring == 1:
        return x_idx.astype(np.int32)
    return None


def compare(semiring, ref, y_idx, y_val, sorted_out=True):
    """Element-wise parity: index sets bit-exact; (min,select2nd) values
    bit-exact; (+,*) values within FP_TOL * sum|a x|.  Returns the largest
    observed |err| / sum|a x| for (+,*)."""
    y_idx = np.asarray(y_idx)
    if sorted_out:
        assert np.all(np.diff(y_idx) > 0), "y_idx not strictly ascending"
        order = np.arange(y_idx.shape[0])
    else:
        order = np.argsort(y_idx, kind="stable")
    np.testing.assert_array_equal(y_idx[order], ref.idx)
    if semiring == 1:
        np.testing.assert_array_equal(np.asarray(y_val)[order], ref.val)
    worst = 0.0
    if semiring == 0:
        err = np.abs(np.asarray(y_val)[order].astype(np.float64) - ref.val)
        scale = np.maximum(ref.absum, np.finfo(np.float64).tiny)
        ratio = err / scale
        bad = ratio > FP_TOL
        assert not bad.any(), "fp32 tolerance exceeded at rows %s (ratio %g)" % (
            ref.idx[bad][:5], ratio.max())
        worst = float(ratio.max(initial=0.0))
    return worst


# ACL (FP32 on the device, FP64 reference): a vertex whose residual came
# within ACL_NEAR (relative) of its threshold eps*d(v) at some step may take
# its push decision the other way in FP32; the FP32 residual's own relative
# error stays below that (a few dozen steps, each adding a handful of
# roundings of 2^-24), so every other decision is the same on both sides.
ACL_NEAR = 1e-4
ACL_TOL = 1e-4  # elementwise, relative to the FP64 value


def acl_compare(p32, r32, colptr, rowidx, seed, alpha, eps, max_steps):
    """Element-wise comparison of one seed's FP32 ACL vectors with the FP64
    trace.  When no vertex came near its threshold, every vertex must agree
    within ACL_TOL.  Otherwise the vertices that disagree must lie within two
    hops of a near vertex (a diverging push moves r(u) ~ eps d(u) to u's
    neighbours, whose own decisions it can move in turn), and their number
    and L1 difference are bounded by what those near vertices hold.
    Returns (number of near vertices, number of disagreeing vertices)."""
    from oracle import acl as oacl
    p64, r64, _, pushes, margin = oacl.acl_trace(colptr, rowidx, seed, alpha, eps, max_steps)
    p32 = np.asarray(p32, np.float64)
    r32 = np.asarray(r32, np.float64)
    floor = 1e-6 * eps  # values this small are rounding residue of zero sums
    bad = (np.abs(p32 - p64) > ACL_TOL * p64 + floor) | (np.abs(r32 - r64) > ACL_TOL * r64 + floor)
    near = np.flatnonzero(margin < ACL_NEAR)
    if near.size == 0:
        assert not bad.any(), "seed %d: %d vertices differ with no near-threshold vertex (e.g. %s)" % (
            seed, int(bad.sum()), np.flatnonzero(bad)[:5])
        return 0, 0
    colptr = np.asarray(colptr, np.int64)
    rowidx = np.asarray(rowidx, np.int64)
    zone = np.zeros(p64.shape[0], bool)
    zone[near] = True
    for _ in range(2):
        idx = np.flatnonzero(zone)
        lens = colptr[idx + 1] - colptr[idx]
        first = np.repeat(colptr[idx] - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens)
        zone[rowidx[first + np.arange(int(lens.sum()))]] = True
    outside = bad & ~zone
    assert not outside.any(), "seed %d: vertices %s differ beyond two hops of the near ones" % (
        seed, np.flatnonzero(outside)[:5])
    deg = np.diff(colptr).astype(np.float64)
    held = float((2.0 * eps * deg[near]).sum())  # about the residual each near vertex holds, twice
    l1 = float(np.abs(p32 - p64)[bad].sum() + np.abs(r32 - r64)[bad].sum())
    assert l1 <= 4.0 * held, "seed %d: L1 difference %g against %g held near threshold" % (
        seed, l1, held)
    return int(near.size), int(bad.sum())
