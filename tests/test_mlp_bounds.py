"""CPU checks of the surrogate's element-wise GPU checks (tests/mlp_bounds.py).

The bf16 rounding helper is pinned against an independent bit-level rounding and hand
values; the exact-grid networks are shown to have one correct result (their fp32 sums
are exact in any order: a float32 BLAS emulation and reordered sums reproduce the fp64
reference bit for bit, and the magnitudes stay below 2^24 grid units); the realistic
tolerances admit a float32 emulation of the kernels and reject planted mistakes (a
dropped K chunk, two swapped output rows, a lost split-K partial)."""
import numpy as np
import pytest

import mlp_bounds as mb
from oracle import mlp as omlp


def test_bf16_rounding_hand_values_and_bit_rounding():
    # ties to even at 1 + 2^-8 (down to 1) and 1 + 3 * 2^-8 (up to 1 + 2^-6); 8 significant bits
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -7, -(1 + 2 ** -8), 255.0, 257.0, 259.0, 0.0,
                  3.0 * 2 ** -130])
    want = np.array([1.0, 1.0, 1 + 2 ** -6, 1 + 2 ** -7, -1.0, 255.0, 256.0, 260.0, 0.0, 3.0 * 2 ** -130])
    assert np.array_equal(mb.bf16_rne(x), want)
    rng = np.random.default_rng(0)
    v = (rng.standard_normal(200_000) * np.exp(rng.uniform(-20, 20, 200_000))).astype(np.float32)
    ties = (np.arange(1, 2001, dtype=np.float32) * np.float32(2 ** -15) + np.float32(2 ** -16)).astype(np.float32)
    for a in (v, ties, -ties):
        assert np.array_equal(mb.bf16_rne(a.astype(np.float64)), mb.bf16_of_f32(a).astype(np.float64))


def test_exact_angles_give_grid_features():
    f = mb.bf16_rne(omlp.features(mb.EXACT_ANGLES[None, :].T.repeat(7, axis=1).astype(np.float64)))
    assert len(mb.EXACT_ANGLES) >= 9
    assert np.all(np.mod(f / mb.G, 1.0) == 0.0)
    assert np.all((f == 0) | (np.abs(f) >= 0.5))


@pytest.mark.parametrize("B", [300, 512, 2048])
def test_exact_grid_networks_have_one_result(B):
    th = mb.exact_network(B)
    q = mb.exact_inputs(B + 1, B)
    r = mb.reference(th, q)
    assert mb.exact_margin_forward(r) < 2.0 ** 23
    y, mask = mb.exact_targets(B + 2, r["out"])
    cnt = mask.sum()
    assert cnt == 2 ** int(np.log2(cnt))
    r = mb.reference(th, q, y, mask)
    assert mb.exact_margin_backward(r, cnt) < 2.0 ** 23.5
    out, loss, flat = mb.emulate_fp32(th, q, y, mask)
    assert np.array_equal(out.astype(np.float64), r["out"])
    assert loss == r["loss"]
    assert np.array_equal(flat.astype(np.float64), r["flat"])
    # another accumulation order (reversed rows) and a two-way split give the same bits
    Wl = [(mb.bf16_of_f32(W.astype(np.float32)), b.astype(np.float32)) for W, b in omlp.unpack(th.astype(np.float64))]
    A = r["acts"][2].astype(np.float32)
    g = r["dz"][2].astype(np.float32)
    rev = g[::-1].T @ A[::-1]
    half = B // 2
    split = (g[:half].T @ A[:half]) + (g[half:].T @ A[half:])
    assert np.array_equal(rev, split) and np.array_equal(rev.astype(np.float64), r["grads"][2][0])
    z = (A[:, ::-1] @ Wl[2][0][:, ::-1].T + Wl[2][1]).astype(np.float64)
    assert np.array_equal(z, r["pre"][2])


def test_exact_grid_catches_planted_mistakes():
    B = 2048
    th = mb.exact_network(B)
    q = mb.exact_inputs(B + 1, B)
    r0 = mb.reference(th, q)
    y, mask = mb.exact_targets(B + 2, r0["out"])
    r = mb.reference(th, q, y, mask)
    for drop in (("kchunk", 2, 5), ("row", 4), ("split",)):
        out, loss, flat = mb.emulate_fp32(th, q, y, mask, drop=drop)
        bad = (out.astype(np.float64) != r["out"]).sum() + (flat.astype(np.float64) != r["flat"]).sum()
        assert bad > 0, drop


@pytest.mark.parametrize("seed,B", [(1, 512), (2, 4096)])
def test_realistic_tolerances_admit_fp32_and_reject_mistakes(seed, B):
    th, q, y, mask = mb.realistic_case(seed, B)
    r = mb.reference(th, q, y, mask)
    S = mb.magnitudes(r)
    out, loss, flat = mb.emulate_fp32(th, q, y, mask)
    assert mb.within(out, r["out"], S["out"], mb.TOL_FWD).all()
    frac, all_ok = mb.grads_ok(flat, r, S)
    assert frac >= mb.GRAD_QUANTILE and all_ok
    assert abs(loss - r["loss"]) <= 2.0 ** -10 * r["loss"]
    # a dropped K chunk in layer 2 of row 5 and swapped output rows leave the bound
    o2, _, f2 = mb.emulate_fp32(th, q, y, mask, drop=("kchunk", 2, 5))
    assert not mb.within(o2, r["out"], S["out"], mb.TOL_FWD).all()
    assert mb.grads_ok(f2, r, S)[0] < 1.0
    o3, _, f3 = mb.emulate_fp32(th, q, y, mask, drop=("row", 4))
    assert (~mb.within(o3, r["out"], S["out"], mb.TOL_FWD)).sum() >= 10
    assert mb.grads_ok(f3, r, S)[0] < 1.0
    if B > 2048:   # a lost split-K partial of every dW
        _, _, f4 = mb.emulate_fp32(th, q, y, mask, drop=("split",))
        assert mb.grads_ok(f4, r, S)[0] < 0.9
