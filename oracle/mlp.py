"""FP64 reference of the schedule-selector network (test infrastructure only).

The same 6 -> 32 -> 32 -> 12 ReLU network and parameter layout as the GPU
selector: W1[32][6] b1[32] W2[32][32] b2[32] W3[12][32] b3[12] mean[6]
scale[6]; inputs are (feature - mean) * scale; the loss is the sum over
samples and valid outputs of the squared error.  Plain numpy, written from
the definition of the network and of back-propagation.
"""
import numpy as np

IN, H, OUT = 6, 32, 12
O_W1 = 0
O_B1 = O_W1 + H * IN
O_W2 = O_B1 + H
O_B2 = O_W2 + H * H
O_W3 = O_B2 + H
O_B3 = O_W3 + OUT * H
NWEIGHT = O_B3 + OUT
O_MEAN = NWEIGHT
O_SCALE = O_MEAN + IN
NPARAM = O_SCALE + IN


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    W1 = p[O_W1:O_B1].reshape(H, IN)
    b1 = p[O_B1:O_W2]
    W2 = p[O_W2:O_B2].reshape(H, H)
    b2 = p[O_B2:O_W3]
    W3 = p[O_W3:O_B3].reshape(OUT, H)
    b3 = p[O_B3:NWEIGHT]
    return W1, b1, W2, b2, W3, b3, p[O_MEAN:O_SCALE], p[O_SCALE:NPARAM]


def forward(p, feats):
    W1, b1, W2, b2, W3, b3, mean, scale = unpack(p)
    x = (np.asarray(feats, np.float64) - mean) * scale
    a1 = x @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    out = h2 @ W3.T + b3
    return out, (x, a1, h1, a2, h2)


def loss_and_grad(p, feats, target, valid=None):
    """Summed squared error over valid outputs and its gradient w.r.t. the
    1676 weights (the normalisation is not trained)."""
    W1, b1, W2, b2, W3, b3, _, _ = unpack(p)
    out, (x, a1, h1, a2, h2) = forward(p, feats)
    v = np.ones_like(out) if valid is None else np.asarray(valid, np.float64)
    diff = (out - np.asarray(target, np.float64)) * v
    loss = float(np.sum(diff * diff))
    d_out = 2.0 * diff
    gW3 = d_out.T @ h2
    gb3 = d_out.sum(axis=0)
    d_h2 = (d_out @ W3) * (a2 > 0)
    gW2 = d_h2.T @ h1
    gb2 = d_h2.sum(axis=0)
    d_h1 = (d_h2 @ W2) * (a1 > 0)
    gW1 = d_h1.T @ x
    gb1 = d_h1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def choose(p, feats, allow_pull=True):
    """Schedule id with the smallest predicted log time (pull = ids 6..11)."""
    out, _ = forward(p, feats)
    if not allow_pull:
        out = out.copy()
        out[..., 6:] = np.inf
    return np.argmin(out, axis=-1)
