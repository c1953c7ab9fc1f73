"""Pins of the FP64 selector-network reference: analytic gradient against
central finite differences, and the forward pass against an explicit loop."""
import numpy as np

from oracle import mlp


def random_problem(seed, n=17):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.4, mlp.NPARAM)
    p[mlp.O_SCALE:] = rng.uniform(0.5, 2.0, mlp.IN)
    feats = rng.normal(0, 2, (n, mlp.IN))
    target = rng.normal(0, 1, (n, mlp.OUT))
    valid = (rng.random((n, mlp.OUT)) < 0.8).astype(np.uint8)
    return p, feats, target, valid


def test_gradient_matches_central_differences():
    p, feats, target, valid = random_problem(1)
    _, g = mlp.loss_and_grad(p, feats, target, valid)
    rng = np.random.default_rng(2)
    idx = rng.choice(mlp.NWEIGHT, size=200, replace=False)
    eps = 1e-6
    for i in idx:
        pp = p.copy(); pp[i] += eps
        pm = p.copy(); pm[i] -= eps
        fd = (mlp.loss_and_grad(pp, feats, target, valid)[0] -
              mlp.loss_and_grad(pm, feats, target, valid)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-4 * max(1.0, abs(fd)), (i, fd, g[i])


def test_forward_matches_explicit_loops():
    p, feats, _, _ = random_problem(3, n=3)
    out, _ = mlp.forward(p, feats)
    W1, b1, W2, b2, W3, b3, mean, scale = mlp.unpack(p)
    for s in range(feats.shape[0]):
        x = [(feats[s][k] - mean[k]) * scale[k] for k in range(6)]
        h1 = [max(0.0, b1[j] + sum(W1[j][k] * x[k] for k in range(6))) for j in range(32)]
        h2 = [max(0.0, b2[j] + sum(W2[j][k] * h1[k] for k in range(32))) for j in range(32)]
        o = [b3[r] + sum(W3[r][k] * h2[k] for k in range(32)) for r in range(12)]
        np.testing.assert_allclose(out[s], o, rtol=1e-12, atol=1e-12)


def test_choose_respects_allow_pull():
    p, feats, _, _ = random_problem(4, n=50)
    c = mlp.choose(p, feats, allow_pull=False)
    assert np.all(c < 6)


def test_forward_on_hand_worked_weights():
    # one path through the network: x -> h1[2] = relu(x0) -> h2[1] = relu(2 h1[2] - 1)
    # -> out[r] = r * h2[1] + b3[r]; the input is normalised as (f - mean) * scale
    p = np.zeros(mlp.NPARAM)
    W1 = p[mlp.O_W1:mlp.O_B1].reshape(mlp.H, mlp.IN)
    W2 = p[mlp.O_W2:mlp.O_B2].reshape(mlp.H, mlp.H)
    W3 = p[mlp.O_W3:mlp.O_B3].reshape(mlp.OUT, mlp.H)
    W1[2, 0] = 1.0
    W2[1, 2] = 2.0
    p[mlp.O_B2 + 1] = -1.0
    W3[:, 1] = np.arange(mlp.OUT)
    p[mlp.O_B3:mlp.NWEIGHT] = 0.5
    p[mlp.O_MEAN:mlp.O_SCALE] = 1.0
    p[mlp.O_SCALE:mlp.NPARAM] = 0.5
    feats = np.array([[4.0, 9, 9, 9, 9, 9],     # x0 = (4-1)*0.5 = 1.5 -> h2[1] = 2
                      [-5.0, 9, 9, 9, 9, 9]])   # x0 = -3 -> h1 = 0 -> h2 = relu(-1) = 0
    out, _ = mlp.forward(p, feats)
    np.testing.assert_allclose(out[0], 2.0 * np.arange(mlp.OUT) + 0.5, rtol=0, atol=1e-15)
    np.testing.assert_allclose(out[1], np.full(mlp.OUT, 0.5), rtol=0, atol=0)
    # squared error against target 0 on outputs 0 and 3 only: 0.5^2 + 6.5^2
    target = np.zeros((1, mlp.OUT))
    valid = np.zeros((1, mlp.OUT), np.uint8)
    valid[0, [0, 3]] = 1
    loss, _ = mlp.loss_and_grad(p, feats[:1], target, valid)
    assert abs(loss - (0.25 + 42.25)) < 1e-12


def test_invalid_outputs_do_not_reach_loss_or_gradient():
    p, feats, target, valid = random_problem(5)
    l0, g0 = mlp.loss_and_grad(p, feats, target, valid)
    t2 = np.where(valid > 0, target, 1e6)
    l1, g1 = mlp.loss_and_grad(p, feats, t2, valid)
    assert l0 == l1 and np.array_equal(g0, g1)
