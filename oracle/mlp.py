"""CPU reference of the learned self-distance surrogate (not in the paper).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Network: features [sin q, cos q] (14) -> 4 x (Linear 256 + ReLU) -> Linear 24, the
per-sphere self-collision distance x_si of Eq. (selftaskvar) in metres.  Loss: mean
squared error over the unmasked (sphere, sample) pairs.  Everything here is float64
numpy; parameters are a flat vector laid out layer by layer as W_l (out x in, row-major)
followed by b_l (out).
"""
from __future__ import annotations

import numpy as np

SIZES = (14, 256, 256, 256, 256, 24)


def n_params(sizes=SIZES) -> int:
    return sum(o * i + o for i, o in zip(sizes[:-1], sizes[1:]))


def unpack(theta, sizes=SIZES):
    out, p = [], 0
    for i, o in zip(sizes[:-1], sizes[1:]):
        W = theta[p:p + o * i].reshape(o, i)
        p += o * i
        b = theta[p:p + o]
        p += o
        out.append((W, b))
    return out


def init_params(seed: int, sizes=SIZES) -> np.ndarray:
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, o in zip(sizes[:-1], sizes[1:]):
        bound = np.sqrt(6.0 / i)
        parts.append(rng.uniform(-bound, bound, size=o * i))
        parts.append(np.zeros(o))
    return np.concatenate(parts)


def features(q):
    q = np.asarray(q, dtype=np.float64)
    return np.concatenate([np.sin(q), np.cos(q)], axis=1)


def forward(theta, q, sizes=SIZES):
    """Returns (output, list of layer inputs) for the backward pass."""
    layers = unpack(theta, sizes)
    a = features(q)
    acts = [a]
    for li, (W, b) in enumerate(layers):
        z = a @ W.T + b
        a = np.maximum(z, 0.0) if li < len(layers) - 1 else z
        acts.append(a)
    return a, acts


def loss_and_grad(theta, q, target, mask=None, sizes=SIZES):
    """Masked MSE and its gradient with respect to theta (backpropagation)."""
    layers = unpack(theta, sizes)
    out, acts = forward(theta, q, sizes)
    m = np.ones_like(out) if mask is None else np.asarray(mask, dtype=np.float64)
    cnt = max(m.sum(), 1.0)
    diff = (out - target) * m
    loss = float((diff * diff).sum() / cnt)
    d = 2.0 * diff / cnt                       # dL / d output
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, b = layers[li]
        a_in = acts[li]
        grads[li] = (d.T @ a_in, d.sum(axis=0))
        if li > 0:
            d = (d @ W) * (acts[li] > 0)       # through the ReLU of the layer below
    g = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, g


def loss_only(theta, q, target, mask=None, sizes=SIZES):
    out, _ = forward(theta, q, sizes)
    m = np.ones_like(out) if mask is None else np.asarray(mask, dtype=np.float64)
    diff = (out - target) * m
    return float((diff * diff).sum() / max(m.sum(), 1.0))


def adamw_step(theta, g, m, v, t, lr, wd, b1=0.9, b2=0.999, eps=1e-8):
    """Decoupled-weight-decay Adam (Loshchilov & Hutter), one step, in place."""
    m[:] = b1 * m + (1 - b1) * g
    v[:] = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    theta[:] = theta - lr * (mh / (np.sqrt(vh) + eps) + wd * theta)
    return theta
