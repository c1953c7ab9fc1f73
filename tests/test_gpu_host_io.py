"""spmspv_run_host (x and y in host memory) against the oracle: every
semiring, both product forms, masks, pinned and pageable buffers, a y
capacity below nnz(y), an empty x, argument checks."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from gpu_util import SEMIRING_TO_ORACLE, compare, mask_bits, need_gpu, x_values

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = need_gpu()
    from paper_1610_07902_gb300 import spmspv as S
    S.load()
    return torch, S


@pytest.fixture(scope="module")
def graph(lib):
    torch, S = lib
    A = synth.rmat(14, seed=31)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val)
    yield A, Ad
    Ad.close()


def host(torch, a, pinned):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.pin_memory() if pinned else t


@pytest.mark.parametrize("semiring", [0, 1, 2])
@pytest.mark.parametrize("nnz_x,masked,pinned", [(300, False, True), (6000, False, True), (6000, True, False),
                                                 (16000, False, False)])
def test_host_buffers_match_oracle(lib, graph, semiring, nnz_x, masked, pinned):
    # 16000 entries of x give W >= 2m: the (+,*) product runs in the direct form
    torch, S = lib
    A, Ad = graph
    xi, xf = synth.frontier(A.n, nnz_x, seed=nnz_x + semiring, stream=2)
    xv = x_values(semiring, xi, xf)
    mask_u8 = (np.random.default_rng(nnz_x).random(A.m) < 0.4).astype(np.uint8) if masked else None
    dmask = torch.from_numpy(mask_bits(mask_u8).view(np.int32)).cuda() if masked else None
    cap = A.m
    yi = host(torch, np.full(cap, -7, np.int32), pinned)
    yv = None if semiring == 2 else host(torch, np.zeros(cap, np.float32 if semiring == 0 else np.int32), pinned)
    k = S.spmspv_run_host(Ad.handle, semiring, host(torch, xi, pinned),
                          None if xv is None else host(torch, xv, pinned), nnz_x, dmask,
                          S.SPMSPV_MASK_COMPLEMENT if masked else 0, yi, yv, cap)
    ref = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, SEMIRING_TO_ORACLE[semiring], xi, xv,
                        mask_u8, True)
    assert k == ref.idx.shape[0]
    compare(semiring, ref, yi.numpy()[:k], None if yv is None else yv.numpy()[:k])
    assert (yi.numpy()[k:k + 8] == -7).all()  # nothing past nnz(y)
    assert S.spmspv_device_status(Ad.handle) == 0


def test_host_capacity_and_empty(lib, graph):
    torch, S = lib
    A, Ad = graph
    xi, xf = synth.frontier(A.n, 4000, seed=5, stream=2)
    ref = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, oracle.PLUS_TIMES, xi, xf)
    cap = 100
    yi = torch.full((cap + 16,), -7, dtype=torch.int32).pin_memory()
    yv = torch.zeros(cap + 16, dtype=torch.float32).pin_memory()
    k = S.spmspv_run_host(Ad.handle, 0, torch.from_numpy(xi).pin_memory(), torch.from_numpy(xf).pin_memory(),
                          xi.size, None, 0, yi, yv, cap)
    assert k == ref.idx.shape[0] > cap
    np.testing.assert_array_equal(yi.numpy()[:cap], ref.idx[:cap])
    assert (yi.numpy()[cap:] == -7).all()
    assert S.spmspv_device_status(Ad.handle) == S.SPMSPV_DEV_CAPACITY
    k = S.spmspv_run_host(Ad.handle, 0, yi, yv, 0, None, 0, yi, yv, cap)
    assert k == 0


def test_host_argument_checks(lib, graph):
    torch, S = lib
    A, Ad = graph
    lib_ = S.load()
    xi = torch.zeros(4, dtype=torch.int32)
    xv = torch.ones(4, dtype=torch.float32)
    y = torch.zeros(8, dtype=torch.int32)
    n = ctypes.c_int32(0)
    stream = S._stream(None)
    # nnz_y NULL, x_val NULL for (+,*), nnz_x beyond n, negative capacity
    assert lib_.spmspv_run_host(Ad.handle, 0, xi.data_ptr(), xv.data_ptr(), 4, None, 0, y.data_ptr(),
                                y.data_ptr(), 8, None, stream) == S.SPMSPV_ERR_ARG
    assert lib_.spmspv_run_host(Ad.handle, 0, xi.data_ptr(), None, 4, None, 0, y.data_ptr(), y.data_ptr(), 8,
                                ctypes.byref(n), stream) == S.SPMSPV_ERR_ARG
    assert lib_.spmspv_run_host(Ad.handle, 0, xi.data_ptr(), xv.data_ptr(), A.n + 1, None, 0, y.data_ptr(),
                                y.data_ptr(), 8, ctypes.byref(n), stream) == S.SPMSPV_ERR_ARG
    assert lib_.spmspv_run_host(Ad.handle, 0, xi.data_ptr(), xv.data_ptr(), 4, None, 0, y.data_ptr(),
                                y.data_ptr(), -1, ctypes.byref(n), stream) == S.SPMSPV_ERR_ARG
