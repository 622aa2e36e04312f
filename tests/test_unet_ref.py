"""Pins of the FP64 reference of the learned guess's network (oracle/unet_ref.py):
the forward convolution against scipy's periodic correlation, the backward
formulas as adjoints, and the whole network's gradient against finite
differences.  No GPU."""
import numpy as np
import pytest

from oracle import unet_ref as U

ndimage = pytest.importorskip("scipy.ndimage")


def _rng(s):
    return np.random.Generator(np.random.PCG64(s))


def test_conv_forward_matches_scipy_wrap_correlation():
    g = _rng(1)
    X = g.standard_normal((6, 6, 6, 3))
    W = g.standard_normal((27, 2, 3))
    b = g.standard_normal(2)
    out = U.conv3_fwd(X, W, b)
    for o in range(2):
        ref = np.full(X.shape[:3], b[o])
        for i in range(3):
            K = W[:, o, i].reshape(3, 3, 3)
            ref += ndimage.correlate(X[..., i], K, mode="wrap")
        np.testing.assert_allclose(out[..., o], ref, rtol=1e-12, atol=1e-12)


def test_conv_backward_are_adjoints():
    g = _rng(2)
    X = g.standard_normal((4, 4, 4, 5))
    W = g.standard_normal((27, 3, 5))
    dZ = g.standard_normal((4, 4, 4, 3))
    lhs = np.sum(U.conv3_fwd(X, W, np.zeros(3)) * dZ)
    assert abs(lhs - np.sum(X * U.conv3_dgrad(dZ, W))) <= 1e-10 * abs(lhs)
    assert abs(lhs - np.sum(W * U.conv3_wgrad(X, dZ))) <= 1e-10 * abs(lhs)


def test_transfers_are_adjoints():
    g = _rng(3)
    x = g.standard_normal((4, 4, 4, 2))
    y = g.standard_normal((8, 8, 8, 2))
    assert abs(np.sum(U.up(x) * y) - np.sum(x * U.up_bwd(y))) <= 1e-12 * np.abs(y).sum()
    assert abs(np.sum(U.pool(y) * x) - np.sum(y * U.pool_bwd(x))) <= 1e-12 * np.abs(y).sum()
    assert np.allclose(U.pool(U.up(x)), x)


def test_network_gradient_matches_finite_differences():
    g = _rng(4)
    P = U.init_params(5)
    for k in P:
        if k.endswith(".b"):
            P[k] = g.standard_normal(P[k].shape) * 0.05  # non-zero biases exercise every path
    X0 = np.zeros((8, 8, 8, 16))
    X0[..., :2] = g.standard_normal((8, 8, 8, 2))
    target = g.standard_normal((8, 8, 8)) * 0.1
    loss, grads, _ = U.loss_and_grads(P, X0, target)
    for name, idx in [("e0.W", (13, 3, 1)), ("e2.W", (4, 10, 7)), ("d2.W", (20, 5, 90)), ("d1.W", (0, 3, 70)),
                      ("d0.W", (26, 15, 40)), ("e3.b", (7,)), ("head", (3,)), ("head", (16,))]:
        eps = 1e-6
        Pp = {k: v.copy() for k, v in P.items()}
        Pm = {k: v.copy() for k, v in P.items()}
        Pp[name][idx] += eps
        Pm[name][idx] -= eps
        fd = (U.loss_and_grads(Pp, X0, target)[0] - U.loss_and_grads(Pm, X0, target)[0]) / (2 * eps)
        an = grads[name][idx]
        assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-8) + 1e-10, (name, idx, fd, an)
