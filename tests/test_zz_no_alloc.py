"""The allocation-free entry point (spmspv_run_noalloc) against the oracle and
against the handle path.

spmspv_run_noalloc serves callers that cannot call cudaMalloc: it keeps its
scratch in one library-owned device array instead of a handle's workspace.
These tests call it through the C ABI at its maximum sizes (m = 2^22 rows,
nnz(A) = 2^20, nnz(x) = 2^16) for every semiring, with and without a mask,
with a y that is too small, and twice in a row (the array keeps the last
call's contents).  This file is named so that pytest collects it last; the
tests pass both in a fresh process and after every other test.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import FP_TOL, compare, mask_bits, need_gpu, x_values

pytestmark = pytest.mark.gpu

M_MAX, NNZ_MAX, X_MAX = 1 << 22, 1 << 20, 1 << 16


def _rect_matrix(m, n, nnz, seed):
    """Seeded random m x n CSC matrix with exactly nnz entries (distinct
    (row, column) pairs, rows ascending in each column), values U[0,1)."""
    rng = np.random.default_rng(seed)
    keys = np.unique(rng.integers(0, m * n, size=int(nnz * 1.02), dtype=np.int64))
    keys = rng.permutation(keys)[:nnz]
    keys.sort()
    col = (keys // m).astype(np.int64)
    row = (keys % m).astype(np.int32)
    colptr = np.concatenate([[0], np.cumsum(np.bincount(col, minlength=n))]).astype(np.int32)
    val = rng.random(nnz, dtype=np.float32)
    return colptr, row, val


@pytest.fixture(scope="module")
def lib():
    torch = need_gpu()
    from paper_1610_07902_gb300 import spmspv as S
    S.load()
    return torch, S


@pytest.fixture(scope="module")
def big(lib):
    torch, S = lib
    m, n = M_MAX, 1 << 18
    colptr, rowidx, val = _rect_matrix(m, n, NNZ_MAX, seed=31)
    d = {k: torch.from_numpy(v).cuda() for k, v in (("colptr", colptr), ("rowidx", rowidx), ("val", val))}
    return m, n, colptr, rowidx, val, d


def _noalloc(torch, S, m, n, d, semiring, x_idx, xv, mask_words, opts, cap):
    yi = torch.full((cap + 64,), -7, dtype=torch.int32, device="cuda")
    yv = torch.full((cap + 64,), -7, dtype=torch.int32, device="cuda")
    nz = torch.zeros(1, dtype=torch.int32, device="cuda")
    xi = torch.from_numpy(x_idx).cuda()
    xvd = None if xv is None else torch.from_numpy(xv).cuda()
    md = None if mask_words is None else torch.from_numpy(mask_words.view(np.int32)).cuda()
    S.spmspv_run_noalloc(m, n, NNZ_MAX, d["colptr"], d["rowidx"], d["val"], S.SPMSPV_VAL_F32,
                         semiring, xi, xvd, x_idx.shape[0], md, opts, yi, yv, cap, nz)
    torch.cuda.synchronize()
    return yi.cpu().numpy(), yv.cpu().numpy(), int(nz.item())


@pytest.mark.parametrize("semiring", [0, 1, 2])
@pytest.mark.parametrize("masking", ["none", "mask", "complement"])
def test_noalloc_at_maximum_size_matches_oracle(lib, big, semiring, masking):
    torch, S = lib
    m, n, colptr, rowidx, val, d = big
    rng = np.random.default_rng(40 + semiring)
    mask = None if masking == "none" else (rng.random(m) < 0.3).astype(np.uint8)
    comp = masking == "complement"
    opts = S.SPMSPV_MASK_COMPLEMENT if comp else 0
    for call in range(2):  # two calls in a row share the scratch array
        x_idx, xf = synth.frontier(n, X_MAX, seed=50 + 10 * semiring + call)
        xv = x_values(semiring, x_idx, xf)
        ref = oracle.spmspv(m, colptr, rowidx, val, {0: oracle.PLUS_TIMES, 1: oracle.MIN_SELECT2ND,
                                                     2: oracle.OR_AND}[semiring],
                            x_idx, xv, mask, comp)
        yi, yv, k = _noalloc(torch, S, m, n, d, semiring, x_idx, xv,
                             None if mask is None else mask_bits(mask), opts, m)
        assert k == ref.idx.shape[0]
        yval = yv[:k].view(np.float32) if semiring == 0 else yv[:k]
        compare(semiring, ref, yi[:k], yval)
        assert (yi[m:] == -7).all() and (yv[m:] == -7).all()  # nothing past y_capacity


def test_noalloc_reports_the_size_a_small_y_needs(lib, big):
    torch, S = lib
    m, n, colptr, rowidx, val, d = big
    x_idx, xf = synth.frontier(n, X_MAX, seed=77)
    ref = oracle.spmspv(m, colptr, rowidx, val, oracle.PLUS_TIMES, x_idx, xf)
    need = ref.idx.shape[0]
    cap = need // 3
    yi, yv, k = _noalloc(torch, S, m, n, d, 0, x_idx, xf, None, 0, cap)
    assert k == need
    # the first cap rows of the sorted y are written, nothing beyond
    np.testing.assert_array_equal(yi[:cap], ref.idx[:cap])
    assert (yi[cap:] == -7).all() and (yv[cap:] == -7).all()


def test_noalloc_matches_handle_path_on_two_calls(lib):
    torch, S = lib
    A = synth.erdos_renyi(60000, d=12, seed=21)          # nnz(A) ~ 720K <= 2^20
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val)
    cap = A.m
    for call, (f, semiring) in enumerate([(3000, S.SPMSPV_PLUS_TIMES_F32),
                                          (20000, S.SPMSPV_PLUS_TIMES_F32)]):
        x_idx, xf = synth.frontier(A.n, f, seed=100 + call)
        xi = torch.from_numpy(x_idx).cuda()
        xv = torch.from_numpy(xf).cuda()
        # the existing entry point (handle with its own workspace)
        yi_h, yv_h, k_h = Ad.multiply(semiring, xi, xv)
        # the allocation-free one
        yi = torch.empty(cap, dtype=torch.int32, device="cuda")
        yv = torch.empty(cap, dtype=torch.float32, device="cuda")
        nz = torch.zeros(1, dtype=torch.int32, device="cuda")
        S.spmspv_run_noalloc(A.m, A.n, A.nnz, Ad.colptr, Ad.rowidx, Ad.val, S.SPMSPV_VAL_F32,
                             semiring, xi, xv, f, None, 0, yi, yv, cap, nz)
        k = int(nz.item())
        assert k == k_h
        np.testing.assert_array_equal(yi[:k].cpu().numpy(), yi_h.cpu().numpy())
        # both within the parity tolerance of the FP64 oracle, so within 2x of each other
        ref = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, oracle.PLUS_TIMES, x_idx, xf)
        diff = np.abs(yv[:k].cpu().numpy().astype(np.float64) - yv_h.cpu().numpy())
        assert np.all(diff <= 2 * FP_TOL * ref.absum)
    Ad.close()


def test_noalloc_rejects_sizes_beyond_its_maximum(lib):
    torch, S = lib
    cp = torch.zeros(2, dtype=torch.int32, device="cuda")
    x = torch.zeros(1, dtype=torch.int32, device="cuda")
    y = torch.zeros(1, dtype=torch.int32, device="cuda")
    nz = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(S.SpmspvError) as e:
        S.spmspv_run_noalloc(M_MAX + 1, 1, 0, cp, None, None, S.SPMSPV_VAL_NONE,
                             S.SPMSPV_OR_AND_BOOL, x, None, 1, None, 0, y, None, 1, nz)
    assert e.value.code == S.SPMSPV_ERR_UNSUPPORTED and "maximum" in str(e.value)
    with pytest.raises(S.SpmspvError) as e:
        S.spmspv_run_noalloc(4, 1, NNZ_MAX + 1, cp, x, None, S.SPMSPV_VAL_NONE,
                             S.SPMSPV_OR_AND_BOOL, x, None, 1, None, 0, y, None, 1, nz)
    assert e.value.code == S.SPMSPV_ERR_UNSUPPORTED and "maximum" in str(e.value)
    xs = torch.zeros(X_MAX + 1, dtype=torch.int32, device="cuda")
    cpn = torch.zeros(X_MAX + 2, dtype=torch.int32, device="cuda")
    with pytest.raises(S.SpmspvError) as e:
        S.spmspv_run_noalloc(4, X_MAX + 1, 0, cpn, None, None, S.SPMSPV_VAL_NONE,
                             S.SPMSPV_OR_AND_BOOL, xs, None, X_MAX + 1, None, 0, y, None, 1, nz)
    assert e.value.code == S.SPMSPV_ERR_UNSUPPORTED and "maximum" in str(e.value)
