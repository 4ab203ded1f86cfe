"""Pins for the surrogate's CPU reference: backpropagation against central differences,
a one-layer closed form, and AdamW's first step."""
import numpy as np
import pytest

from oracle import mlp


def test_gradient_matches_central_differences():
    sizes = (14, 9, 7, 5)
    rng = np.random.default_rng(0)
    theta = mlp.init_params(1, sizes) + rng.normal(scale=0.05, size=mlp.n_params(sizes))
    q = rng.uniform(-np.pi, np.pi, size=(6, 7))
    y = rng.normal(size=(6, 5))
    mask = (rng.random((6, 5)) < 0.8).astype(float)
    _, g = mlp.loss_and_grad(theta, q, y, mask, sizes)
    idx = rng.choice(theta.size, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        num = (mlp.loss_only(theta + e, q, y, mask, sizes) - mlp.loss_only(theta - e, q, y, mask, sizes)) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(num)), (i, num, g[i])


def test_single_linear_layer_closed_form():
    """One linear layer: L = mean((W f + b - y)^2) so dL/dW = 2/N (W f + b - y) f^T."""
    sizes = (14, 3)
    rng = np.random.default_rng(3)
    theta = rng.normal(size=mlp.n_params(sizes))
    q = rng.uniform(-3, 3, size=(4, 7))
    y = rng.normal(size=(4, 3))
    W = theta[:42].reshape(3, 14)
    b = theta[42:]
    f = np.concatenate([np.sin(q), np.cos(q)], axis=1)
    r = f @ W.T + b - y
    loss, g = mlp.loss_and_grad(theta, q, y, None, sizes)
    assert np.isclose(loss, (r ** 2).sum() / r.size)
    assert np.allclose(g[:42].reshape(3, 14), 2 * r.T @ f / r.size)
    assert np.allclose(g[42:], 2 * r.sum(axis=0) / r.size)


def test_adamw_first_step_is_sign_step():
    """With bias correction, Adam's first update is lr * sign(g) (|g| >> eps), plus decay."""
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m, v = np.zeros(3), np.zeros(3)
    out = mlp.adamw_step(theta.copy(), g, m, v, 1, lr=0.01, wd=0.1)
    assert np.allclose(out, theta - 0.01 * (np.sign(g) + 0.1 * theta), atol=1e-6)
