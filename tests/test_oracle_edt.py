"""Pins for the oracle's EDT (Sec. III-C, Alg. 1): the oracle is checked against things
other than itself -- scipy's independent EDT, the definition by brute force, closed
forms for one and two sites, and invariants every exact EDT satisfies."""
import numpy as np
import pytest
from scipy import ndimage

from paper_2407_02363_b300 import synth

INT32_MAX = np.iinfo(np.int32).max


def _coords(lin, dims):
    X, Y, Z = dims
    lin = np.asarray(lin, dtype=np.int64)
    return lin % X, (lin // X) % Y, lin // (X * Y)


def _check_idx_valid(occ, sq, ix):
    """Every index names an occupied voxel at exactly the reported squared distance."""
    Z, Y, X = occ.shape
    flat = occ.reshape(-1)
    if not flat.any():
        assert (sq == INT32_MAX).all() and (ix == -1).all()
        return
    ixf = ix.reshape(-1).astype(np.int64)
    assert (ixf >= 0).all() and (ixf < occ.size).all()
    assert flat[ixf].all()
    vx, vy, vz = _coords(np.arange(occ.size), (X, Y, Z))
    sx, sy, sz = _coords(ixf, (X, Y, Z))
    d = (vx - sx) ** 2 + (vy - sy) ** 2 + (vz - sz) ** 2
    assert np.array_equal(d, sq.reshape(-1).astype(np.int64))


def _scipy_sqdist(occ):
    """Integer squared distance from scipy's nearest-feature indices (independent EDT)."""
    _, ind = ndimage.distance_transform_edt(occ == 0, return_indices=True)
    Z, Y, X = occ.shape
    gz, gy, gx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    return ((gz - ind[0]) ** 2 + (gy - ind[1]) ** 2 + (gx - ind[2]) ** 2).astype(np.int64)


@pytest.mark.parametrize("density", [0.002, 0.02, 0.1, 0.5])
@pytest.mark.parametrize("seed", range(5))
def test_brute_matches_scipy_16(oracle_mod, density, seed):
    occ = synth.random_occupancy(seed, (16, 16, 16), density)
    if not occ.any():
        occ[3, 5, 7] = 1
    sq, ix = oracle_mod.edt_brute(occ)
    assert np.array_equal(sq.astype(np.int64), _scipy_sqdist(occ).reshape(-1))
    _check_idx_valid(occ, sq.reshape(occ.shape), ix.reshape(occ.shape))


@pytest.mark.parametrize("seed", range(100))
def test_separable_matches_brute_16(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    density = float(10 ** rng.uniform(-3, np.log10(0.5)))
    occ = synth.random_occupancy(1000 + seed, (16, 16, 16), density)
    sq, ix = oracle_mod.edt(occ)
    bsq, _ = oracle_mod.edt_brute(occ)
    assert np.array_equal(sq.reshape(-1), bsq)
    _check_idx_valid(occ, sq, ix)


@pytest.mark.parametrize("dims", [(24, 16, 8), (7, 13, 5), (33, 1, 9), (1, 1, 40), (40, 3, 1)])
def test_separable_matches_scipy_anisotropic(oracle_mod, dims):
    occ = synth.random_occupancy(sum(dims), dims, 0.03)
    if not occ.any():
        occ.reshape(-1)[len(occ.reshape(-1)) // 2] = 1
    sq, ix = oracle_mod.edt(occ)
    assert np.array_equal(sq.astype(np.int64), _scipy_sqdist(occ))
    _check_idx_valid(occ, sq, ix)


@pytest.mark.parametrize("seed", range(6))
def test_single_site_closed_form(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    dims = tuple(int(v) for v in rng.integers(1, 40, 3))
    site = tuple(int(rng.integers(0, d)) for d in dims)
    occ = synth.sites_occupancy(dims, [site])
    sq, ix = oracle_mod.edt(occ)
    Z, Y, X = occ.shape
    gz, gy, gx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    expect = (gx - site[0]) ** 2 + (gy - site[1]) ** 2 + (gz - site[2]) ** 2
    assert np.array_equal(sq, expect)
    assert (ix == site[0] + X * (site[1] + Y * site[2])).all()


def test_two_sites_closed_form(oracle_mod):
    dims = (30, 20, 10)
    a, b = (3, 4, 5), (25, 17, 2)
    occ = synth.sites_occupancy(dims, [a, b])
    sq, ix = oracle_mod.edt(occ)
    Z, Y, X = occ.shape
    gz, gy, gx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    da = (gx - a[0]) ** 2 + (gy - a[1]) ** 2 + (gz - a[2]) ** 2
    db = (gx - b[0]) ** 2 + (gy - b[1]) ** 2 + (gz - b[2]) ** 2
    assert np.array_equal(sq, np.minimum(da, db))
    _check_idx_valid(occ, sq, ix)


def test_empty_map(oracle_mod):
    occ = np.zeros((6, 5, 4), dtype=np.uint8)
    sq, ix = oracle_mod.edt(occ)
    assert (sq == INT32_MAX).all() and (ix == -1).all()
    bsq, bix = oracle_mod.edt_brute(occ)
    assert (bsq == INT32_MAX).all() and (bix == -1).all()


def test_full_map(oracle_mod):
    occ = np.ones((5, 6, 7), dtype=np.uint8)
    sq, ix = oracle_mod.edt(occ)
    assert (sq == 0).all()
    assert np.array_equal(ix.reshape(-1), np.arange(occ.size))


def test_one_dimensional_row(oracle_mod):
    """Y = Z = 1: the EDT is the squared distance to the nearest occupied position."""
    rng = np.random.default_rng(7)
    row = (rng.random(300) < 0.03).astype(np.uint8)
    row[[0, 299]] = 0
    row[150] = 1
    occ = row.reshape(1, 1, -1)
    sq, _ = oracle_mod.edt(occ)
    sites = np.flatnonzero(row)
    expect = [min((i - s) ** 2 for s in sites) for i in range(row.size)]
    assert np.array_equal(sq.reshape(-1), np.array(expect))


def _lipschitz_ok(sq, axis):
    """sqrt(Dp) <= sqrt(Dq) + 1 for 6-neighbours, in integers:
    Dp > Dq  =>  (Dp - Dq - 1)^2 <= 4 Dq."""
    a = sq.astype(np.int64)
    p = np.moveaxis(a, axis, 0)[1:]
    q = np.moveaxis(a, axis, 0)[:-1]
    for P, Q in ((p, q), (q, p)):
        m = P > Q
        lhs = (P - Q - 1)[m]
        assert ((lhs < 0) | (lhs * lhs <= 4 * Q[m])).all()


def test_invariants_scene_64(oracle_mod):
    grid = synth.GridSpec((64, 64, 64), 0.02)
    pts = synth.surface_cloud(1234 + 1000, grid)
    occ = np.zeros((64, 64, 64), dtype=np.uint8)
    oracle_mod.insert_points(occ, None, grid.dims, grid.voxel_size, grid.origin, pts)
    assert occ.any()
    sq, ix = oracle_mod.edt(occ)
    assert np.array_equal(sq == 0, occ != 0)
    _check_idx_valid(occ, sq, ix)
    for ax in range(3):
        _lipschitz_ok(sq, ax)
    # D is at most the squared distance along the row alone
    for z in range(0, 64, 9):
        for y in range(0, 64, 7):
            row = np.flatnonzero(occ[z, y])
            if row.size:
                d1 = np.min((np.arange(64)[:, None] - row[None, :]) ** 2, axis=1)
                assert (sq[z, y] <= d1).all()
    # scipy agrees on the whole grid
    assert np.array_equal(sq.astype(np.int64), _scipy_sqdist(occ))


def test_brute_sampled_matches_separable_128(oracle_mod):
    occ = synth.random_occupancy(99, (128, 96, 80), 0.001)
    sq, _ = oracle_mod.edt(occ)
    rng = np.random.default_rng(3)
    q = rng.integers(0, occ.size, 3000)
    bsq, bix = oracle_mod.edt_brute(occ, q)
    assert np.array_equal(sq.reshape(-1)[q], bsq)


def _golden_cases():
    import glob
    import json
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    for p in sorted(glob.glob(os.path.join(here, "*.json"))):
        with open(p) as f:
            yield os.path.basename(p), json.load(f)


@pytest.mark.parametrize("name,case", list(_golden_cases()))
def test_golden_fixtures(oracle_mod, name, case):
    X, Y, Z = case["dims"]
    occ = synth.sites_occupancy((X, Y, Z), [tuple(s) for s in case["sites"]])
    sq, ix = oracle_mod.edt(occ)
    assert np.array_equal(sq, np.array(case["sqdist_zyx"], dtype=np.int64))
    _check_idx_valid(occ, sq, ix)
