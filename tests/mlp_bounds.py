"""References and element-wise bounds for the surrogate's bf16 tensor-core kernels.

Test infrastructure.  The fp64 oracle (`oracle.mlp`) fixes what the network computes.
The kernels compute it with bf16 operands and fp32 accumulation and round at fixed
points: the features and every hidden activation to bf16 (after bias and ReLU), the
output gradient 2 (out - y) m / count and every backpropagated gradient to bf16.  This
module provides two element-wise checks of the kernels against that definition.

1. Exact-grid networks (bit-exact).  Joint angles are drawn from the angles whose sine
   and cosine are 0, +-1 or have magnitude >= 1/2 (multiples of pi/6 and pi/4, never
   pi/2 or pi, where the fp32 angle gives a tiny non-zero value), so every bf16 feature
   is a multiple of G = 2^-8.  Weights are small integers and biases multiples of G, so
   every pre-activation is a multiple of G, and every bf16 rounding of such a value is a
   multiple of G again.  As long as the sum of the magnitudes of a dot product's terms is
   below 2^24 units of its grid, fp32 holds every partial sum exactly, in any order and
   with any split, so the kernels' result has exactly one correct value: the fp64
   reference with the same rounding points.  Targets y = out - delta with delta on a
   2^-2 grid and a mask with a power-of-two count make the gradients and the loss exact
   the same way.
   `exact_margin_*` verify that precondition for every entry.

2. Realistic networks (He-initialised dense weights).  Here the fp32 accumulation order
   decides some bf16 roundings: an activation whose pre-activation lies within the
   accumulation error (about 2^-20 relative) of a rounding boundary comes out one bf16
   ulp (at most 2^-7 relative) away from the reference's, and that difference reaches
   the later layers.  So the check is element-wise against magnitudes: |got - ref| <=
   tol * S, with S the sum of |terms| of the entry's own dot product (for a gradient
   entry, with every backpropagated gradient replaced by the |terms| sum it came from;
   `magnitudes`).  Forward outputs: every entry within tol = 2^-7.  Gradients: a ReLU
   whose pre-activation rounds to zero on one side only switches a whole backpropagated
   term, so at least 99.9 % of the entries within 2^-7 and every entry within 2^-2.  A
   wrong output row, a dropped 16-wide K chunk or a missed split-K partial moves entries
   by percents of S (tests/test_mlp_bounds.py plants such mistakes in an fp32 CPU
   emulation and checks both directions).
"""
from __future__ import annotations

import numpy as np

from oracle import mlp as omlp

G = 2.0 ** -8            # grid of the exact networks' activations
TOL_FWD = 2.0 ** -7          # every forward output
TOL_GRAD = 2.0 ** -7         # at least GRAD_QUANTILE of the gradient entries
TOL_GRAD_ALL = 2.0 ** -2     # every gradient entry
GRAD_QUANTILE = 0.999


def bf16_rne(x):
    """Round float64 values to the bfloat16 grid, to nearest, ties to even."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                     # x = m 2^e, 0.5 <= |m| < 1
    scale = np.ldexp(1.0, e - 8)           # bf16 keeps 8 significant bits
    return np.where(x == 0.0, 0.0, np.round(x / scale) * scale)


def bf16_of_f32(x):
    """Round float32 values to bfloat16 (to nearest even), as float32."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


# ------------------------------------------------------------------ reference
def reference(theta, q, y=None, mask=None):
    """fp64 forward (and backward if y is given) with the kernels' rounding points.

    Returns a dict: acts (layer inputs, bf16 values), pre (pre-activations), out,
    and with y: loss, dz (per layer: the gradient at that layer's output, bf16), grads
    (per layer (dW, db)), flat (gradients in the oracle's parameter order)."""
    layers = [(bf16_rne(W), np.asarray(b, np.float64)) for W, b in omlp.unpack(np.asarray(theta, np.float64))]
    q = np.asarray(q, np.float32).astype(np.float64)
    a = bf16_rne(omlp.features(q))
    acts, pre = [a], []
    for li, (W, b) in enumerate(layers):
        z = a @ W.T + b
        pre.append(z)
        if li < len(layers) - 1:
            a = bf16_rne(np.maximum(z, 0.0))
            acts.append(a)
    out = z
    r = {"layers": layers, "acts": acts, "pre": pre, "out": out}
    if y is None:
        return r
    y = np.asarray(y, np.float32).astype(np.float64)
    m = np.ones_like(y) if mask is None else np.asarray(mask, np.float64)
    cnt = max(float(m.sum()), 1.0)
    d = (out - y) * m
    r["loss"] = float((d * d).sum() / cnt)
    g = bf16_rne(2.0 * d / cnt)
    dz = [None] * len(layers)
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        dz[li] = g
        grads[li] = (g.T @ acts[li], g.sum(axis=0))
        if li > 0:
            g = bf16_rne((g @ W) * (acts[li] > 0))
    r["dz"], r["grads"] = dz, grads
    r["flat"] = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return r


def magnitudes(r):
    """Per entry, the magnitude its rounding differences scale with: for a forward output
    the sum of |terms| of its dot product; for a gradient entry the same sum with every
    backpropagated gradient replaced by the |terms| sum that produced it (so an entry
    whose gradient input came from a cancelling sum gets that sum's scale, not its small
    value).  Returned as {"out": [B, 24], "flat": oracle parameter order}."""
    layers, acts = r["layers"], r["acts"]
    S = {"out": np.abs(acts[-1]) @ np.abs(layers[-1][0]).T + np.abs(layers[-1][1])}
    if "grads" in r:
        parts = [None] * len(layers)
        Mg = np.abs(r["dz"][-1])
        for li in range(len(layers) - 1, -1, -1):
            parts[li] = np.concatenate([(Mg.T @ np.abs(acts[li])).ravel(), Mg.sum(axis=0)])
            if li > 0:
                Mg = (Mg @ np.abs(layers[li][0])) * (acts[li] > 0)
        S["flat"] = np.concatenate(parts)
    return S


def within(got, ref, S, tol):
    """Boolean mask of entries with |got - ref| <= tol * S (plus an fp32 ulp of ref)."""
    got = np.asarray(got, np.float64)
    slack = tol * S + 2.0 ** -23 * np.abs(ref) + 1e-30
    return np.abs(got - ref) <= slack


# ------------------------------------------------------------------ exact-grid networks
def _exact_angles():
    """fp32 angles whose sine and cosine round to bf16 values on the 2^-8 grid, with the
    fp64 sine / cosine of the fp32 angle at least 2^-16 (relative) away from a bf16
    rounding boundary, far beyond sinf's error."""
    cands = [0.0] + [s * k * np.pi / 6 for k in (1, 2, 4, 5) for s in (1, -1)] + \
            [s * k * np.pi / 4 for k in (1, 3) for s in (1, -1)]
    keep = []
    for c in cands:
        q = np.float32(c)
        ok = True
        for v in (np.sin(np.float64(q)), np.cos(np.float64(q))):
            r = bf16_rne(v)
            if abs(r) not in (0.0, 1.0) and not (abs(r) >= 0.5 and abs(r) < 1.0):
                ok = False
            if v != 0.0 and abs(v) != 1.0:
                m, e = np.frexp(abs(v))
                frac = (abs(v) / np.ldexp(1.0, e - 8)) % 1.0   # position between bf16 values
                if abs(frac - 0.5) < 2.0 ** -16 * 256:
                    ok = False
            if not float(r / G).is_integer():
                ok = False
        if ok:
            keep.append(q)
    return np.array(keep, dtype=np.float32)


EXACT_ANGLES = _exact_angles()


def exact_network(seed, nnz=(3, 3, 3, 3), w0=1):
    """Integer weights (layer 0 in [-w0, w0], later layers nnz[l - 1] entries of +-1 per row)
    and biases on the 2^-8 grid, as a flat fp32 parameter vector."""
    rng = np.random.default_rng(seed)
    parts = []
    for li, (i, o) in enumerate(zip(omlp.SIZES[:-1], omlp.SIZES[1:])):
        if li == 0:
            W = rng.integers(-w0, w0 + 1, size=(o, i)).astype(np.float64)
        else:
            W = np.zeros((o, i))
            k = nnz[li - 1]
            for row in range(o):
                cols = rng.choice(i, size=k, replace=False)
                W[row, cols] = rng.choice([-1.0, 1.0], size=k)
        b = rng.integers(-64, 129, size=o) * G
        parts += [W.ravel(), b]
    return np.concatenate(parts).astype(np.float32)


def exact_inputs(seed, B):
    rng = np.random.default_rng(seed)
    return rng.choice(EXACT_ANGLES, size=(B, 7)).astype(np.float32)


def exact_targets(seed, out, frac=2.0 / 3.0):
    """y = out - delta (delta in {0, +-1/4, +-1/2}) and a 0/1 mask with a power-of-two
    number of ones (about `frac` of the entries)."""
    rng = np.random.default_rng(seed)
    delta = rng.choice([0.0, 0.25, -0.25, 0.5, -0.5], size=out.shape)
    y = (out - delta).astype(np.float32)
    assert np.array_equal(y.astype(np.float64), out - delta)
    n = out.size
    cnt = 1 << int(np.floor(np.log2(max(frac * n, 1))))
    mask = np.zeros(n, np.float32)
    mask[rng.choice(n, size=cnt, replace=False)] = 1.0
    return y, mask.reshape(out.shape)


def _units(x, grid):
    return np.abs(x) / grid


def exact_margin_forward(r):
    """Largest |term| sum of any forward dot product, in units of its grid (2^-8 times
    the weights' integer grid); must stay below 2^24 for exact fp32 sums."""
    worst = 0.0
    for li, (W, b) in enumerate(r["layers"]):
        S = np.abs(r["acts"][li]) @ np.abs(W).T + np.abs(b)
        worst = max(worst, float(_units(S, G).max()))
        assert np.all(np.mod(r["pre"][li] / G, 1.0) == 0.0)
    return worst


def exact_margin_backward(r, cnt):
    """Largest |term| sum of any backward dot product in units of its grid
    (gradients on the grid 2^-2 * 2 / count)."""
    gd = 2.0 ** -2 * 2.0 / cnt
    worst = 0.0
    for li in range(len(r["layers"])):
        g = r["dz"][li]
        assert np.all(np.mod(g / gd, 1.0) == 0.0)
        worst = max(worst, float(_units(np.abs(g).T @ np.abs(r["acts"][li]), gd * G).max()))
        worst = max(worst, float(_units(np.abs(g).sum(axis=0), gd).max()))
        if li > 0:
            worst = max(worst, float(_units(np.abs(g) @ np.abs(r["layers"][li][0]), gd).max()))
    return worst


# ------------------------------------------------------------------ fp32 CPU emulation
def emulate_fp32(theta, q, y=None, mask=None, drop=None):
    """The kernels' computation in float32 numpy (BLAS accumulation order), used by the
    CPU tests of these checks.  `drop` plants a mistake: ("kchunk", layer, row) leaves
    out K columns [16, 32) of that layer for that row; ("row", layer) swaps the first two
    output rows; ("split",) loses the second 1024-row chunk of every dW."""
    layers = [(bf16_of_f32(W.astype(np.float32)), b.astype(np.float32))
              for W, b in omlp.unpack(np.asarray(theta, np.float64))]
    q = np.asarray(q, np.float32)
    a = bf16_of_f32(np.concatenate([np.sin(q), np.cos(q)], axis=1))
    acts = [a]
    for li, (W, b) in enumerate(layers):
        z = (a @ W.T + b).astype(np.float32)
        if drop and drop[0] == "kchunk" and drop[1] == li:
            row = drop[2]
            z[row] = (a[row, :16] @ W[:, :16].T + a[row, 32:] @ W[:, 32:].T + b).astype(np.float32)
        if drop and drop[0] == "row" and drop[1] == li:
            z[[0, 1]] = z[[1, 0]]
        if li < len(layers) - 1:
            a = bf16_of_f32(np.maximum(z, 0.0))
            acts.append(a)
    out = z
    if y is None:
        return out
    m = np.ones_like(out) if mask is None else np.asarray(mask, np.float32)
    cnt = np.float32(max(float(m.sum()), 1.0))
    d = ((out - y) * m).astype(np.float32)
    g = bf16_of_f32((np.float32(2.0) * d) / cnt)
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        A = acts[li]
        if drop and drop[0] == "split" and g.shape[0] > 1024:
            dW = g[:1024].T @ A[:1024] + g[2048:].T @ A[2048:]
        else:
            dW = g.T @ A
        grads[li] = (dW.astype(np.float32), g.sum(axis=0, dtype=np.float32))
        if li > 0:
            g = bf16_of_f32((g @ W) * (A > 0))
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return out, float((d * d).sum() / cnt), flat


def grads_ok(got_flat, r, S):
    """(fraction of gradient entries within TOL_GRAD, all entries within TOL_GRAD_ALL)."""
    frac = float(np.mean(within(got_flat, r["flat"], S["flat"], TOL_GRAD)))
    return frac, bool(within(got_flat, r["flat"], S["flat"], TOL_GRAD_ALL).all())


def realistic_case(seed, B):
    """He-initialised parameters perturbed by N(0, 0.02), uniform joint angles, targets in
    [0, 1] m and a mask keeping about 85 % of the entries."""
    rng = np.random.default_rng(seed)
    theta = (omlp.init_params(seed % 97) + rng.normal(scale=0.02, size=omlp.n_params())).astype(np.float32)
    q = rng.uniform(-np.pi, np.pi, size=(B, 7)).astype(np.float32)
    y = rng.uniform(0.0, 1.0, size=(B, 24)).astype(np.float32)
    mask = (rng.random((B, 24)) < 0.85).astype(np.float32)
    return theta, q, y, mask
