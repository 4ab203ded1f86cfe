"""Pins of the statistical-outlier-filter oracle (Sec. III-A) against things it does not
compute itself: closed forms on a lattice, a planted-outlier cloud, an independent k-d
tree, numpy's mean / standard deviation, invariance under permutation, edge cases."""
import math

import numpy as np
import pytest

from oracle import sor


def lattice(n, s):
    g = np.arange(n, dtype=np.float32) * np.float32(s)
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def test_lattice_closed_forms():
    """Cubic lattice with spacing s = 2^-6 (exact in float32): an interior point's six
    nearest neighbours are at s; a corner's three at s and three at s*sqrt(2); an edge
    point (not a corner) has four at s and two at s*sqrt(2)."""
    s = 2.0 ** -6
    p = lattice(5, s)
    d, valid = sor.mean_knn_distance(p, 6)
    assert valid.all()
    idx = lambda i, j, k: (i * 5 + j) * 5 + k
    assert d[idx(2, 2, 2)] == s                               # exact: sqrt(2^-12) = 2^-6
    assert math.isclose(d[idx(0, 0, 0)], (3 * s + 3 * s * math.sqrt(2)) / 6, rel_tol=1e-15)
    assert math.isclose(d[idx(0, 0, 2)], (4 * s + 2 * s * math.sqrt(2)) / 6, rel_tol=1e-15)
    # k = 1: every lattice point's nearest neighbour is at s
    d1, _ = sor.mean_knn_distance(p, 1)
    assert (d1 == s).all()


def test_planted_outliers_are_exactly_the_dropped_points():
    rng = np.random.default_rng(0)
    cluster = rng.normal(0, 0.05, (2000, 3)).astype(np.float32)
    far = (rng.uniform(-1, 1, (6, 3)) * 20 + 40).astype(np.float32)
    p = np.concatenate([cluster, far])
    keep, d, (mean, std, thr) = sor.sor_filter(p, 20, 1.0)
    assert keep[-6:].sum() == 0
    assert keep[:-6].all()
    assert (d[-6:] > thr).all()


def test_knn_means_match_an_independent_kdtree():
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(1)
    p = rng.uniform(-1, 1, (3000, 3)).astype(np.float32)
    for k in (1, 8, 50):
        d, _ = sor.mean_knn_distance(p, k)
        dist, _ = spatial.cKDTree(p.astype(np.float64)).query(p.astype(np.float64), k=k + 1)
        ref = dist[:, 1:].mean(axis=1)
        np.testing.assert_allclose(d, ref, rtol=1e-12, atol=0)


def test_statistics_match_numpy_mean_and_sample_std():
    rng = np.random.default_rng(2)
    dv = rng.uniform(0.001, 0.5, 5000)
    mean, std, thr = sor.threshold(dv, 1.5)
    assert math.isclose(mean, dv.mean(), rel_tol=1e-13)
    assert math.isclose(std, dv.std(ddof=1), rel_tol=1e-9)
    assert thr == mean + 1.5 * std


def test_permutation_invariance():
    rng = np.random.default_rng(3)
    p = np.concatenate([rng.normal(0, 0.1, (1500, 3)), rng.uniform(-3, 3, (40, 3))]).astype(np.float32)
    keep, d, st = sor.sor_filter(p, 10, 1.0)
    perm = rng.permutation(len(p))
    keep2, d2, st2 = sor.sor_filter(p[perm], 10, 1.0)
    assert np.array_equal(keep2, keep[perm])
    assert np.array_equal(d2, d[perm])
    assert st2 == st


def test_edge_cases():
    nan = np.float32(np.nan)
    # invalid points are dropped and ignored
    p = np.array([[0, 0, 0], [nan, 0, 0], [1, 0, 0], [0, np.inf, 0]], np.float32)
    keep, d, _ = sor.sor_filter(p, 5, 1.0)
    assert list(keep) == [1, 0, 1, 0]
    assert d[0] == 1.0 and d[2] == 1.0 and np.isnan(d[1])
    # one valid point: d = 0, kept
    keep, d, st = sor.sor_filter(np.array([[1, 2, 3]], np.float32), 4, 1.0)
    assert list(keep) == [1] and d[0] == 0.0 and st == (0.0, 0.0, 0.0)
    # duplicates: a point's copy is its nearest neighbour at distance 0
    p = np.array([[0, 0, 0], [0, 0, 0], [3, 0, 0]], np.float32)
    d, _ = sor.mean_knn_distance(p, 1)
    assert list(d) == [0.0, 0.0, 3.0]
    # no valid point
    keep, d, st = sor.sor_filter(np.full((3, 3), nan, np.float32), 2, 1.0)
    assert keep.sum() == 0 and all(math.isnan(v) for v in st)


def test_fixed_point_sums_do_not_depend_on_order():
    rng = np.random.default_rng(4)
    dv = rng.uniform(0, 2, 1000)
    a = sor.threshold(dv, 1.0)
    b = sor.threshold(dv[::-1].copy(), 1.0)
    assert a == b
