"""Pins of the start-vector network oracle (oracle/warmstart.py).

* the 3x3 convolution against scipy's 2D cross-correlation, channel by
  channel (an independent library routine);
* pooling and upsampling on small arrays written out by hand;
* the subspace-capture loss: 0 for u in span(Q), 1 for u orthogonal to it,
  and its gradient by central differences;
* the gradient of the whole network by central differences on a 32 x 32
  input, along random directions and per layer (step 1e-7; the ReLU kinks
  make larger steps less accurate; absolute slack 2e-9, the rounding of a
  difference of two losses L ~ 1 divided by the step);
* a planted mistake in the backward pass (the pooling adjoint scaled by 1/2
  instead of 1/4) fails the difference check;
* one Adam step from zero moments moves each parameter by lr * sign(g).
"""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import warmstart as W


def test_conv3x3_matches_scipy_cross_correlation():
    rng = np.random.default_rng(0)
    z = rng.standard_normal((3, 11, 9))
    Wt = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = W.conv3x3(z, Wt, b)
    for o in range(4):
        ref = b[o] + sum(correlate2d(z[c], Wt[o, c], mode="same", boundary="fill") for c in range(3))
        assert np.allclose(y[o], ref, atol=1e-13)


def test_pool_and_up_by_hand():
    z = np.arange(16.0).reshape(1, 4, 4)
    assert np.array_equal(W.pool(z)[0], [[2.5, 4.5], [10.5, 12.5]])
    assert np.array_equal(W.up(np.array([[[1.0, 2.0]]]))[0], [[1, 1, 2, 2], [1, 1, 2, 2]])
    g = np.ones((1, 2, 2))
    assert np.array_equal(W.pool_backward(g)[0], np.full((4, 4), 0.25))
    assert np.array_equal(W.up_backward(np.ones((1, 4, 4)))[0], np.full((2, 2), 4.0))
    # adjoints: <P z, g> = <z, P^T g>, <U z, g> = <z, U^T g>
    rng = np.random.default_rng(1)
    z, g = rng.standard_normal((2, 6, 8)), rng.standard_normal((2, 3, 4))
    assert abs(np.sum(W.pool(z) * g) - np.sum(z * W.pool_backward(g))) < 1e-13
    assert abs(np.sum(W.up(g) * z) - np.sum(g * W.up_backward(z))) < 1e-13


def test_loss_values_and_gradient():
    rng = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rng.standard_normal((64, 5)))
    u_in = (Q @ rng.standard_normal(5)).reshape(8, 8)
    assert abs(W.loss(u_in, Q)[0]) < 1e-14
    v = rng.standard_normal(64)
    u_out = (v - Q @ (Q.T @ v)).reshape(8, 8)
    assert abs(W.loss(u_out, Q)[0] - 1.0) < 1e-14
    u = rng.standard_normal((8, 8))
    L, g = W.loss(u, Q)
    d = rng.standard_normal((8, 8))
    eps = 1e-6
    fd = (W.loss(u + eps * d, Q)[0] - W.loss(u - eps * d, Q)[0]) / (2 * eps)
    assert abs(fd - np.sum(g * d)) < 1e-9
    # scale invariance: dL/du is orthogonal to u
    assert abs(np.sum(g * u)) < 1e-12


def _setup(seed=0, H=32, Wd=32, q=4):
    rng = np.random.default_rng(seed)
    theta = rng.standard_normal(sum(W.param_sizes())) * 0.1
    x = rng.standard_normal((3, H, Wd))
    Q, _ = np.linalg.qr(rng.standard_normal((H * Wd, q)))
    return theta, x, Q


def _fd(theta, x, Q, v, eps=1e-7):
    Lp = W.loss(W.forward(theta + eps * v, x)[0], Q)[0]
    Lm = W.loss(W.forward(theta - eps * v, x)[0], Q)[0]
    return (Lp - Lm) / (2 * eps)


def test_network_gradient_by_central_differences():
    theta, x, Q = _setup()
    L, g, _ = W.loss_and_grad(theta, x, Q)
    assert 0.0 <= L <= 1.0
    rng = np.random.default_rng(10)
    for _ in range(3):
        v = rng.standard_normal(theta.size)
        assert abs(_fd(theta, x, Q, v) - g @ v) <= 1e-6 * abs(g @ v) + 2e-9
    sizes = W.param_sizes()
    off = np.concatenate([[0], np.cumsum(sizes)])
    for slot in (0, 1, 4, 13, 16, 28, 29):          # W1, b1, W3, b7, W9, W15, b15
        v = np.zeros(theta.size)
        v[off[slot]:off[slot + 1]] = rng.standard_normal(sizes[slot])
        assert abs(_fd(theta, x, Q, v) - g @ v) <= 1e-6 * abs(g @ v) + 2e-9, slot


def test_planted_pool_adjoint_mistake_is_caught(monkeypatch):
    theta, x, Q = _setup(seed=3)
    monkeypatch.setattr(W, "pool_backward", lambda g: np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) / 2.0)
    L, g, _ = W.loss_and_grad(theta, x, Q)
    sizes = W.param_sizes()
    v = np.zeros(theta.size)
    v[:sizes[0]] = np.random.default_rng(4).standard_normal(sizes[0])   # W1 sees the pooled paths
    assert abs(_fd(theta, x, Q, v) - g @ v) > 1e-3 * abs(_fd(theta, x, Q, v))


def test_adam_first_step_moves_by_lr_sign():
    rng = np.random.default_rng(5)
    th = rng.standard_normal(100)
    g = rng.standard_normal(100)
    m, v = np.zeros(100), np.zeros(100)
    th0 = th.copy()
    W.adam(th, m, v, g, 1, 1e-3)
    assert np.allclose(th0 - th, 1e-3 * np.sign(g), rtol=1e-6, atol=0)
