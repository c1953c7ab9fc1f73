"""The learned schedule selector on the GPU.

- its hand-written gradient kernel against the FP64 reference (oracle/mlp.py)
- training with its own kernels lowers the loss
- the device-side choice equals the reference network's argmin on the
  features the device computed
- any choice leaves results unchanged (spmspv_run and BFS, SPMSPV_SCHED_AUTO)
"""
import numpy as np
import pytest

import oracle
from oracle import mlp
import synth
from gpu_util import SEMIRING_TO_ORACLE, compare, need_gpu, x_values

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = need_gpu()
    from paper_1610_07902_gb300 import spmspv as S
    S.load()
    return torch, S


def random_params(seed):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.3, mlp.NPARAM).astype(np.float32)
    p[mlp.O_MEAN:mlp.O_SCALE] = rng.normal(0, 1, 6)
    p[mlp.O_SCALE:] = rng.uniform(0.2, 1.0, 6)
    return p


def test_gradient_matches_fp64_reference(lib):
    torch, S = lib
    A = synth.rmat(10, seed=1)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val)
    p = random_params(3)
    S.spmspv_selector_set(Ad.handle, p)
    rng = np.random.default_rng(4)
    n = 300
    feats = rng.normal(0, 3, (n, 6)).astype(np.float32)
    target = rng.normal(0, 2, (n, 12)).astype(np.float32)
    valid = (rng.random((n, 12)) < 0.7).astype(np.uint8)
    g, loss = S.spmspv_selector_grad(Ad.handle, torch.from_numpy(feats).cuda(),
                                     torch.from_numpy(target).cuda(), torch.from_numpy(valid).cuda(), n)
    ref_loss, ref_g = mlp.loss_and_grad(p.astype(np.float64), feats, target, valid)
    assert abs(loss - ref_loss) <= 1e-4 * abs(ref_loss)
    np.testing.assert_allclose(g, ref_g, rtol=0, atol=1e-4 * np.abs(ref_g).max())
    Ad.close()


def test_training_lowers_the_loss(lib):
    torch, S = lib
    A = synth.rmat(10, seed=1)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val)
    teacher = random_params(7).astype(np.float64)
    rng = np.random.default_rng(8)
    feats = rng.normal(0, 2, (2000, 6)).astype(np.float32)
    target = mlp.forward(teacher, feats)[0].astype(np.float32)
    loss = S.spmspv_selector_train(Ad.handle, torch.from_numpy(feats).cuda(),
                                   torch.from_numpy(target).cuda(), None, 2000, 60, 64, 3e-3, 1)
    assert np.all(np.isfinite(loss))
    assert loss[-1] < 0.3 * loss[0]
    Ad.close()


def test_device_choice_matches_reference_and_results_unchanged(lib):
    torch, S = lib
    A = synth.rmat(13, seed=3)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
    rng = np.random.default_rng(9)
    for seed in range(6):
        p = random_params(100 + seed)
        S.spmspv_selector_set(Ad.handle, p)
        for f in [3, 400, 5000]:
            x_idx, xf = synth.frontier(A.n, f, seed=seed * 10 + f)
            mask = (rng.random(A.m) < 0.5).astype(np.uint8)
            for semiring in (1, 2):
                from test_gpu_spmspv import _run
                xv = x_values(semiring, x_idx, xf)
                yi, yv, k, st = _run(lib, A, Ad, semiring, x_idx, xv, mask, True, None, auto=True)
                assert st == 0
                ref = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, SEMIRING_TO_ORACLE[semiring],
                                    x_idx, xv, mask, True)
                compare(semiring, ref, yi, yv)
                feats = S.spmspv_last_features(Ad.handle)
                assert abs(feats[3] - mask.mean()) < 1e-6
                chosen = S.spmspv_last_schedule(Ad.handle)
                want = int(mlp.choose(p.astype(np.float64), feats[None, :].astype(np.float64))[0])
                out = mlp.forward(p.astype(np.float64), feats[None, :].astype(np.float64))[0][0]
                # ties within float rounding may go either way
                assert chosen == want or abs(out[chosen] - out[want]) < 1e-4
        # BFS with the learned schedule: identical levels and parents
        src = int(synth.sources(A.colptr, 1, seed=seed)[0])
        lv, par, nl, _, _ = oracle.bfs(A.colptr, A.rowidx, src)
        level, parent, nlv = Ad.bfs(src, S.SPMSPV_SCHED_AUTO)
        np.testing.assert_array_equal(level.cpu().numpy(), lv)
        np.testing.assert_array_equal(parent.cpu().numpy(), par)
        assert nlv == nl
    Ad.close()


def test_device_features_match_their_definition(lib):
    """The six features the selector evaluates on the device, against their
    definition computed on the host from the same x, mask and matrix:
    log2(1+f), log2(1+W), the degree skew max_k d_k / (W / fc) with fc the x
    entries whose column is non-empty, the mask density, log2 m and nnz/n."""
    torch, S = lib
    from test_gpu_spmspv import _run
    A = synth.rmat(14, seed=4)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
    S.spmspv_selector_set(Ad.handle, random_params(7))
    deg = np.diff(A.colptr).astype(np.int64)
    rng = np.random.default_rng(11)
    for f in [1, 37, 2000, 9000]:
        x_idx, xf = synth.frontier(A.n, f, seed=f)
        for masked in (False, True):
            mask = (rng.random(A.m) < 0.35).astype(np.uint8) if masked else None
            for semiring in (0, 1):
                xv = x_values(semiring, x_idx, xf)
                _, _, _, st = _run(lib, A, Ad, semiring, x_idx, xv, mask, True, None, auto=True)
                assert st == 0
                got = S.spmspv_last_features(Ad.handle).astype(np.float64)
                d = deg[x_idx]
                W, fc = int(d.sum()), int((d > 0).sum())
                want = np.array([np.log2(1 + f), np.log2(1 + W),
                                 d.max() * fc / W if W else 0.0,
                                 mask.sum() / A.m if masked else 0.0,
                                 np.log2(A.m), A.nnz / A.n])
                np.testing.assert_allclose(got, want, rtol=2e-6, atol=1e-7,
                                           err_msg="f=%d masked=%s semiring=%d" % (f, masked, semiring))
    Ad.close()


def test_selector_load_reads_the_weights_file(lib, tmp_path):
    """spmspv_selector_load installs the parameters of a weights file, the
    same ones spmspv_selector_set installs from an array; a malformed file is
    refused and leaves the installed parameters unchanged."""
    torch, S = lib
    from paper_1610_07902_gb300 import selector
    A = synth.rmat(10, seed=2)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val)
    S.spmspv_selector_load(Ad.handle, selector.WEIGHTS)
    np.testing.assert_array_equal(S.spmspv_selector_get(Ad.handle), selector.load()[0])
    bad = tmp_path / "short.json"
    bad.write_text('{"nparam": 3, "params": [1.0, 2.0, 3.0]}')
    with pytest.raises(S.SpmspvError) as e:
        S.spmspv_selector_load(Ad.handle, bad)
    assert e.value.code == S.SPMSPV_ERR_ARG
    with pytest.raises(S.SpmspvError):
        S.spmspv_selector_load(Ad.handle, tmp_path / "missing.json")
    np.testing.assert_array_equal(S.spmspv_selector_get(Ad.handle), selector.load()[0])
    Ad.close()


def test_unmasked_auto_call_stays_push(lib):
    """Weights that rate every pull schedule fastest: a masked call pulls, an
    unmasked one keeps to the push schedules (the network was never trained on
    unmasked calls, whose pull would read every row), both exact."""
    torch, S = lib
    A = synth.rmat(13, seed=5)
    Ad = S.CscMatrix(A.m, A.n, A.colptr, A.rowidx, A.val, flags=S.SPMSPV_CSC_PATTERN_SYMMETRIC)
    p = random_params(7)
    p[mlp.O_B3 + 6:mlp.O_B3 + 12] = -100.0  # the pull schedules' output biases
    S.spmspv_selector_set(Ad.handle, p)
    from test_gpu_spmspv import _run
    x_idx, xf = synth.frontier(A.n, 500, seed=3)
    mask = (np.random.default_rng(4).random(A.m) < 0.5).astype(np.uint8)
    for use_mask in (True, False):
        yi, yv, k, st = _run(lib, A, Ad, 1, x_idx, x_idx.astype(np.int32), mask if use_mask else None, True,
                             None, auto=True)
        assert st == 0
        ref = oracle.spmspv(A.m, A.colptr, A.rowidx, A.val, SEMIRING_TO_ORACLE[1], x_idx, x_idx.astype(np.int32),
                            mask if use_mask else None, True)
        compare(1, ref, yi, yv)
        chosen = S.spmspv_last_schedule(Ad.handle)
        assert (chosen >= 6) == use_mask, (use_mask, chosen)
    Ad.close()
