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
