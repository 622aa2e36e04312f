"""Plain FP64 numpy reference of the learned initial guess's network: 3x3x3
periodic convolutions, 2x2x2 mean pooling, nearest-neighbour upsampling,
channel concatenation, ReLU, a 1x1x1 output head and the squared-error loss,
with their gradients written out from the definitions.

TEST INFRASTRUCTURE ONLY (gradient checks of the CUDA kernels).  The paper has
no learned component; this file is the definition the tensor-core kernels are
checked against.

Layout: a field is an array [n, n, n, C] (voxel-major, channels last); a
3x3x3 kernel is W[27, cout, cin], tap t = (di+1)*9 + (dj+1)*3 + (dk+1) for the
offset (di, dj, dk) in {-1,0,1}^3, periodic:
    out[v, o] = b[o] + sum_t sum_i X[v + d_t, i] W[t, o, i]
"""
from __future__ import annotations

import numpy as np

TAPS = [(di, dj, dk) for di in (-1, 0, 1) for dj in (-1, 0, 1) for dk in (-1, 0, 1)]


def shift(X, d):
    """Y[v] = X[v + d] with periodic wrap (X: [n, n, n, C])."""
    return np.roll(X, shift=(-d[0], -d[1], -d[2]), axis=(0, 1, 2))


def conv3_fwd(X, W, b):
    out = np.zeros(X.shape[:3] + (W.shape[1],))
    for t, d in enumerate(TAPS):
        out += shift(X, d) @ W[t].T
    return out + b


def conv3_dgrad(dZ, W):
    """d/dX of sum(out * dZ): dX[u] = sum_t dZ[u - d_t] W[t]."""
    dX = np.zeros(dZ.shape[:3] + (W.shape[2],))
    for t, d in enumerate(TAPS):
        dX += shift(dZ, (-d[0], -d[1], -d[2])) @ W[t]
    return dX


def conv3_wgrad(X, dZ):
    """dW[t, o, i] = sum_v dZ[v, o] X[v + d_t, i]."""
    n3 = X.shape[0] * X.shape[1] * X.shape[2]
    Z = dZ.reshape(n3, -1)
    return np.stack([Z.T @ shift(X, d).reshape(n3, -1) for d in TAPS])


def pool(X):
    n = X.shape[0] // 2
    return X.reshape(n, 2, n, 2, n, 2, -1).mean(axis=(1, 3, 5))


def pool_bwd(dY):
    return np.repeat(np.repeat(np.repeat(dY, 2, 0), 2, 1), 2, 2) / 8.0


def up(X):
    return np.repeat(np.repeat(np.repeat(X, 2, 0), 2, 1), 2, 2)


def up_bwd(dY):
    n = dY.shape[0] // 2
    return dY.reshape(n, 2, n, 2, n, 2, -1).sum(axis=(1, 3, 5))


def relu(x):
    return np.maximum(x, 0.0)


# ---------------------------------------------------------------------------
# The network: 4 levels, channels (16, 32, 64, 64), skip connections by
# concatenation, nearest upsampling, mean pooling, ReLU, 1x1x1 head.
# ---------------------------------------------------------------------------

# (name, cin pieces, cout): the encoder e0..e3 and decoder d2..d0
LAYERS = [("e0", (16,), 16), ("e1", (16,), 32), ("e2", (32,), 64), ("e3", (64,), 64),
          ("d2", (64, 64), 64), ("d1", (64, 32), 32), ("d0", (32, 16), 16)]


def init_params(seed: int = 0):
    """He-normal weights, zero biases; head weights small."""
    rng = np.random.Generator(np.random.PCG64(seed))
    P = {}
    for name, pieces, cout in LAYERS:
        cin = sum(pieces)
        P[name + ".W"] = rng.standard_normal((27, cout, cin)) * np.sqrt(2.0 / (27 * cin))
        P[name + ".b"] = np.zeros(cout)
    P["head"] = np.concatenate([rng.standard_normal(16) * 0.1, [0.0]])
    return P


def forward(P, X0):
    """X0: [n, n, n, 16] input features.  Returns (prediction [n,n,n], cache)."""
    c = {"x0": X0}
    c["e0"] = relu(conv3_fwd(X0, P["e0.W"], P["e0.b"]))
    c["p0"] = pool(c["e0"])
    c["e1"] = relu(conv3_fwd(c["p0"], P["e1.W"], P["e1.b"]))
    c["p1"] = pool(c["e1"])
    c["e2"] = relu(conv3_fwd(c["p1"], P["e2.W"], P["e2.b"]))
    c["p2"] = pool(c["e2"])
    c["e3"] = relu(conv3_fwd(c["p2"], P["e3.W"], P["e3.b"]))
    c["in_d2"] = np.concatenate([up(c["e3"]), c["e2"]], axis=-1)
    c["d2"] = relu(conv3_fwd(c["in_d2"], P["d2.W"], P["d2.b"]))
    c["in_d1"] = np.concatenate([up(c["d2"]), c["e1"]], axis=-1)
    c["d1"] = relu(conv3_fwd(c["in_d1"], P["d1.W"], P["d1.b"]))
    c["in_d0"] = np.concatenate([up(c["d1"]), c["e0"]], axis=-1)
    c["d0"] = relu(conv3_fwd(c["in_d0"], P["d0.W"], P["d0.b"]))
    pred = c["d0"] @ P["head"][:16] + P["head"][16]
    return pred, c


def loss_and_grads(P, X0, target):
    """Mean squared error of the prediction and the gradient of every parameter."""
    pred, c = forward(P, X0)
    V = pred.size
    r = pred - target
    loss = float(np.mean(r * r))
    g = {}
    dpred = 2.0 * r / V
    g["head"] = np.concatenate([np.tensordot(dpred, c["d0"], axes=3), [dpred.sum()]])
    dd0 = dpred[..., None] * P["head"][:16]

    def layer_bwd(name, X, Y, dY):
        dZ = dY * (Y > 0)
        g[name + ".W"] = conv3_wgrad(X, dZ)
        g[name + ".b"] = dZ.sum(axis=(0, 1, 2))
        return conv3_dgrad(dZ, P[name + ".W"])

    dx = layer_bwd("d0", c["in_d0"], c["d0"], dd0)
    dd1, de0 = up_bwd(dx[..., :32]), dx[..., 32:]
    dx = layer_bwd("d1", c["in_d1"], c["d1"], dd1)
    dd2, de1 = up_bwd(dx[..., :64]), dx[..., 64:]
    dx = layer_bwd("d2", c["in_d2"], c["d2"], dd2)
    de3, de2 = up_bwd(dx[..., :64]), dx[..., 64:]
    dp2 = layer_bwd("e3", c["p2"], c["e3"], de3)
    de2 = de2 + pool_bwd(dp2)
    dp1 = layer_bwd("e2", c["p1"], c["e2"], de2)
    de1 = de1 + pool_bwd(dp1)
    dp0 = layer_bwd("e1", c["p0"], c["e1"], de1)
    de0 = de0 + pool_bwd(dp0)
    layer_bwd("e0", c["x0"], c["e0"], de0)
    return loss, g, pred
