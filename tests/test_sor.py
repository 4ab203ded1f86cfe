"""GPU parity of the statistical outlier filter (Sec. III-A) against the brute-force CPU
oracle: per-point mean kNN distances, the cloud statistics and every keep decision
bit-equal; the masked insert equals the oracle's insert of the kept points."""
import numpy as np
import pytest
import torch

import oracle
from oracle import sor
from paper_2407_02363_b300 import synth
from gpu_helpers import lib

pytestmark = pytest.mark.gpu


def run_gpu(p, k, std_mul, f=None):
    v = lib()
    own = f is None
    if own:
        f = v.OutlierFilter(max(len(p), 1))
    x = torch.from_numpy(np.ascontiguousarray(p, np.float32)).cuda()
    keep = torch.empty(len(p), dtype=torch.uint8, device="cuda")
    f.filter(x, keep, k=k, std_mul=std_mul)
    stats, counts = f.stats()
    d = f.mean_distances(len(p)).clone().cpu().numpy() if len(p) else np.zeros(0)
    if own:
        f.close()
    return keep.cpu().numpy(), d, stats, counts


def assert_parity(p, k, std_mul, f=None):
    keep, d, stats, counts = run_gpu(p, k, std_mul, f)
    okeep, od, ostats = sor.sor_filter(p, k, std_mul)
    valid = np.isfinite(np.asarray(p, np.float32)).all(axis=1)
    assert np.array_equal(d[valid], od[valid]), f"{int((d[valid] != od[valid]).sum())} distances differ"
    assert np.array_equal(keep, okeep), f"{int((keep != okeep).sum())} decisions differ"
    if valid.any():
        assert stats == ostats
    assert counts == (int(valid.sum()), int(okeep.sum()))
    return keep


def cloud(seed, n, n_out=20):
    rng = np.random.default_rng(seed)
    a = rng.normal(0, 0.05, (n // 2, 3)) + [0.3, 0.2, 0.1]
    b = np.stack([rng.uniform(-0.5, 0.5, n - n // 2), rng.uniform(-0.5, 0.5, n - n // 2),
                  rng.normal(0, 0.003, n - n // 2)], axis=1)      # a noisy plane
    o = rng.uniform(-2, 2, (n_out, 3))
    return np.concatenate([a, b, o]).astype(np.float32)


@pytest.mark.parametrize("k,std_mul", [(1, 1.0), (8, 0.5), (50, 1.0), (64, 2.0)])
def test_random_clouds(k, std_mul):
    assert_parity(cloud(10 + k, 6000), k, std_mul)


def test_camera_scene_cloud_and_reuse_of_one_filter():
    v = lib()
    g = synth.GridSpec((128, 128, 128), 0.02)
    f = v.OutlierFilter(30_000)
    for i in range(2):
        p = synth.CameraScene(5 + i, g, n_points=12_000 + 8_000 * i).frame(i)
        assert_parity(p, 50, 1.0, f)
    f.close()


def test_lattice_ties_duplicates_and_invalid_points():
    s = np.float32(2.0 ** -6)
    gr = np.arange(12, dtype=np.float32) * s
    x, y, z = np.meshgrid(gr, gr, gr, indexing="ij")
    p = np.stack([x.ravel(), y.ravel(), z.ravel()], 1)
    p = np.concatenate([p, p[:50], [[np.nan, 0, 0], [0, np.inf, 1], [5, 5, 5]]]).astype(np.float32)
    assert_parity(p, 6, 1.0)
    assert_parity(p, 26, 0.0)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 5])
def test_tiny_clouds(n):
    rng = np.random.default_rng(n)
    p = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    keep, d, stats, counts = run_gpu(p, 10, 1.0)
    okeep, od, ostats = sor.sor_filter(p, 10, 1.0)
    assert np.array_equal(keep, okeep)
    assert counts == (n, int(okeep.sum()))
    if n:
        assert np.array_equal(d, od) and stats == ostats


def test_identical_points_and_far_outliers_widen_the_grid():
    rng = np.random.default_rng(7)
    same = np.zeros((300, 3), np.float32)
    far = rng.uniform(-50, 50, (8, 3)).astype(np.float32)
    near = rng.normal(0, 0.01, (2000, 3)).astype(np.float32)
    assert_parity(np.concatenate([same, near, far]), 16, 1.0)
    assert_parity(np.zeros((40, 3), np.float32), 8, 1.0)


def test_masked_insert_equals_oracle_insert_of_kept_points():
    v = lib()
    g = synth.GridSpec((96, 96, 96), 0.02)
    p = synth.CameraScene(21, g, n_points=15_000).frame(0)
    p = np.concatenate([p, np.random.default_rng(1).uniform(0, 1.9, (300, 3)).astype(np.float32)])
    keep = assert_parity(p, 30, 1.0)
    m = v.Map(g.dims, g.voxel_size, g.origin)
    m.clear(v.MAP_BOTH)
    x = torch.from_numpy(p).cuda()
    kd = torch.from_numpy(keep).cuda()
    m.insert_pointcloud_masked(x, kd)
    got = m.occupancy(v.MAP_ENV).cpu().numpy()
    env = np.zeros((96, 96, 96), np.uint8)
    slf = np.zeros_like(env)
    oracle.insert_points(env, slf, g.dims, g.voxel_size, g.origin, p[keep.astype(bool)])
    assert np.array_equal(got, env)
    m.close()


def test_rejects_bad_arguments():
    v = lib()
    f = v.OutlierFilter(100)
    x = torch.zeros((101, 3), dtype=torch.float32, device="cuda")
    keep = torch.empty(101, dtype=torch.uint8, device="cuda")
    for kw in ({"k": 0}, {"k": 65}, {"std_mul": float("nan")}):
        with pytest.raises(v.VedtError):
            f.filter(x, keep, n=100, **kw)
    with pytest.raises(v.VedtError):
        f.filter(x, keep, n=101)
    f.close()
