"""Pins for the oracle's insertion (Alg. 2 lines 5-7, Sec. III-A), sphere query
(Eq. (dist), Alg. 3 lines 3-4) and forward kinematics: hand-placed points with
hand-computed voxels, exact binary-fraction poses, closed-form planar kinematics, and
float64 geometry for the query."""
import math

import numpy as np
import pytest

from paper_2407_02363_b300 import synth


def _grid(dims):
    X, Y, Z = dims
    return np.zeros((Z, Y, X), dtype=np.uint8)


def test_points_hand_placed(oracle_mod):
    dims, vs, org = (4, 4, 4), 0.1, (0.0, 0.0, 0.0)
    pts = np.array([
        [0.05, 0.05, 0.05],      # voxel (0,0,0)
        [0.1, 0.0, 0.0],         # lower face of voxel (1,0,0): 0.1f/0.1f == 1
        [0.4, 0.0, 0.0],         # upper face of the grid: 0.4f/0.1f == 4 -> outside
        [-1e-7, 0.2, 0.2],       # just below the origin -> floor = -1 -> outside
        [np.nan, 0.1, 0.1],      # NaN -> dropped
        [0.35, 0.25, 0.15],      # voxel (3,2,1)
    ], dtype=np.float32)
    env = _grid(dims)
    n = oracle_mod.insert_points(env, None, dims, vs, org, pts)
    assert n == 3
    assert set(zip(*np.nonzero(env))) == {(0, 0, 0), (0, 0, 1), (1, 2, 3)}  # (z, y, x)


def test_points_origin_and_transform(oracle_mod):
    dims, vs, org = (8, 8, 8), 0.5, (-2.0, -2.0, -2.0)
    # translation by exactly (+1.0, -0.5, +2.0): binary fractions, so the voxel is exact
    T = np.array([[1, 0, 0, 1.0], [0, 1, 0, -0.5], [0, 0, 1, 2.0]], dtype=np.float32)
    pts = np.array([[-1.75, 0.25, -3.75]], dtype=np.float32)
    env = _grid(dims)
    assert oracle_mod.insert_points(env, None, dims, vs, org, pts, T=T) == 1
    # world (-0.75, -0.25, -1.75) -> ((w+2)/0.5) = (2.5, 3.5, 0.5) -> voxel (2, 3, 0)
    assert set(zip(*np.nonzero(env))) == {(0, 3, 2)}


def test_points_robot_filter(oracle_mod):
    dims, vs, org = (4, 4, 4), 0.25, (0.0, 0.0, 0.0)
    self_map = _grid(dims)
    self_map[1, 1, 1] = 1
    pts = np.array([[0.3, 0.3, 0.3], [0.6, 0.6, 0.6]], dtype=np.float32)
    env = _grid(dims)
    assert oracle_mod.insert_points(env, self_map, dims, vs, org, pts, filter_self=True) == 1
    assert set(zip(*np.nonzero(env))) == {(2, 2, 2)}
    env2 = _grid(dims)
    assert oracle_mod.insert_points(env2, self_map, dims, vs, org, pts, filter_self=False) == 2


def test_points_counting_invariant(oracle_mod):
    grid = synth.GridSpec((64, 64, 64), 0.02)
    pts = synth.surface_cloud(7, grid, n_points=5000)
    env = _grid(grid.dims)
    n = oracle_mod.insert_points(env, None, grid.dims, grid.voxel_size, grid.origin, pts)
    assert 0 < int(env.sum()) <= n <= len(pts)


def test_links_exact_poses(oracle_mod):
    dims, vs, org = (8, 8, 8), 0.5, (0.0, 0.0, 0.0)
    link = np.array([[0.25, 0.25, 0.25], [0.75, 0.25, 0.25], [0.25, 1.25, 0.75]], dtype=np.float32)
    ident = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], dtype=np.float32)
    # rotation by +90 deg about z (exact in fp32) then translation (2, 1, 0.5)
    rot = np.array([[0, -1, 0, 2.0], [1, 0, 0, 1.0], [0, 0, 1, 0.5]], dtype=np.float32)
    s = _grid(dims)
    n = oracle_mod.insert_links(s, dims, vs, org, [link, link], np.stack([ident, rot]), 0b11)
    assert n == 6
    # identity: voxels (0,0,0), (1,0,0), (0,2,1)
    # rotated: (x,y,z) -> (2 - y, 1 + x, 0.5 + z):
    #   (0.25,0.25,0.25) -> (1.75, 1.25, 0.75) -> voxel (3, 2, 1)
    #   (0.75,0.25,0.25) -> (1.75, 1.75, 0.75) -> voxel (3, 3, 1)
    #   (0.25,1.25,0.75) -> (0.75, 1.25, 1.25) -> voxel (1, 2, 2)
    expect = {(0, 0, 0), (0, 0, 1), (1, 2, 0), (1, 2, 3), (1, 3, 3), (2, 2, 1)}  # (z,y,x)
    assert set(zip(*np.nonzero(s))) == expect
    s2 = _grid(dims)
    oracle_mod.insert_links(s2, dims, vs, org, [link, link], np.stack([ident, rot]), 0b10)
    assert set(zip(*np.nonzero(s2))) == {(1, 2, 3), (1, 3, 3), (2, 2, 1)}


def test_fk_planar_closed_form(oracle_mod):
    """All joint axes parallel to world z, links along x: the frame origin of link k is
    sum_{i<k} L_i (cos th_i, sin th_i) with th_i = q_1 + ... + q_i."""
    n = 5
    L = [0.3, 0.25, 0.2, 0.15, 0.1]
    base = np.zeros((3, 4)); base[:, :3] = np.eye(3); base[:, 3] = (0.1, -0.2, 0.7)
    offs = np.zeros((n, 3, 4))
    for k in range(n):
        offs[k, :, :3] = np.eye(3)
        offs[k, :, 3] = (L[k - 1] if k > 0 else 0.0, 0.0, 0.0)
    chain = synth.Chain(base=base, offsets=offs, lengths=np.array(L))
    q = np.array([0.3, -1.1, 2.0, 0.7, -0.4])
    P = oracle_mod.fk(chain, q)
    th = np.cumsum(q)
    for k in range(1, n + 1):
        x = 0.1 + sum(L[i] * math.cos(th[i]) for i in range(k - 1))
        y = -0.2 + sum(L[i] * math.sin(th[i]) for i in range(k - 1))
        assert abs(P[k, 0, 3] - x) < 1e-12 and abs(P[k, 1, 3] - y) < 1e-12
        assert abs(P[k, 2, 3] - 0.7) < 1e-12
        R = P[k, :, :3]
        assert np.allclose(R, [[math.cos(th[k - 1]), -math.sin(th[k - 1]), 0],
                               [math.sin(th[k - 1]), math.cos(th[k - 1]), 0], [0, 0, 1]], atol=1e-12)


def _planar_chain(L, base_xyz, base_R=None):
    """All joint axes parallel to the base's z axis, link k+1 offset along link k's x."""
    n = len(L)
    base = np.zeros((3, 4))
    base[:, :3] = np.eye(3) if base_R is None else base_R
    base[:, 3] = base_xyz
    offs = np.zeros((n, 3, 4))
    for k in range(n):
        offs[k, :, :3] = np.eye(3)
        offs[k, :, 3] = (L[k - 1] if k > 0 else 0.0, 0.0, 0.0)
    return synth.Chain(base=base, offsets=offs, lengths=np.array(L))


@pytest.mark.parametrize("tilt", [False, True])
def test_sphere_centres_planar_closed_form(oracle_mod, tilt):
    """Alg. 2 line 8 on a planar chain, by hand: link k's frame has heading
    th_k = q_1 + ... + q_k and origin p_k = b + sum_{i<k} L_i (cos th_i, sin th_i, 0); a
    sphere at local (lx, ly, lz) on link k sits at
    p_k + (lx cos th_k - ly sin th_k, lx sin th_k + ly cos th_k, lz).
    Off-axis local offsets, every link, the static body (link 0, th_0 = 0) and a base
    tilted 90 degrees about x (the plane becomes x-z) catch a wrong link index, a
    transposed rotation and a dropped translation."""
    L = [0.3, 0.25, 0.2, 0.15, 0.1]
    b = np.array([0.1, -0.2, 0.7])
    Rb = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, -1.0], [0.0, 1.0, 0.0]]) if tilt else np.eye(3)
    chain = _planar_chain(L, b, Rb)
    rng = np.random.default_rng(17)
    links = np.array([0, 1, 1, 2, 3, 3, 4, 5, 5, 2], dtype=np.int32)
    local = rng.uniform(-0.1, 0.1, size=(len(links), 3))
    sph = synth.SphereModel(link=links, local=local, radius=np.full(len(links), 0.05, np.float32))
    for q in (np.array([0.3, -1.1, 2.0, 0.7, -0.4]), rng.uniform(-np.pi, np.pi, 5)):
        got = oracle_mod.sphere_centres(chain, sph, q)
        th = np.concatenate([[0.0], np.cumsum(q)])          # th[k] = heading of link k
        org = [np.zeros(3)]
        for k in range(1, len(L) + 1):
            o = np.zeros(3)
            for i in range(1, k):
                o += L[i - 1] * np.array([math.cos(th[i]), math.sin(th[i]), 0.0])
            org.append(o)
        for i, (k, (lx, ly, lz)) in enumerate(zip(links, local)):
            c, s_ = math.cos(th[k]), math.sin(th[k])
            planar = org[k] + np.array([lx * c - ly * s_, lx * s_ + ly * c, lz])
            want = b + Rb @ planar
            assert np.abs(got[i].astype(np.float64) - want).max() <= 1e-6, (i, k, got[i], want)


def test_fk_rotations_orthonormal(oracle_mod):
    chain = synth.make_chain(5, (1.0, 1.0, 1.0))
    for q in synth.joint_states(6, 10):
        P = oracle_mod.fk(chain, q)
        for T in P:
            R = T[:, :3]
            assert np.allclose(R @ R.T, np.eye(3), atol=1e-12)
            assert abs(np.linalg.det(R) - 1) < 1e-12
        # link k+1's origin lies at distance L_k from link k's origin along link k's z axis
        for k in range(1, chain.n_joints):
            d = P[k + 1, :, 3] - P[k, :, 3]
            assert np.allclose(d, chain.lengths[k - 1] * P[k, :, 2], atol=1e-12)


def test_query_single_site_geometry(oracle_mod):
    dims, vs, org = (20, 16, 12), 0.02, (0.1, -0.3, 0.05)
    site = (13, 2, 9)
    occ = synth.sites_occupancy(dims, [site])
    sq, ix = oracle_mod.edt(occ)
    rng = np.random.default_rng(11)
    vox = np.stack([rng.integers(0, d, 40) for d in dims], axis=1)
    c = (np.asarray(org) + (vox + rng.uniform(0.1, 0.9, vox.shape)) * vs).astype(np.float32)
    r = np.full(len(c), 0.05, dtype=np.float32)
    out = oracle_mod.query_spheres(sq, ix, dims, vs, org, c, r)
    for i in range(len(c)):
        v = np.floor((c[i].astype(np.float64) - org) / vs).astype(int)
        d = vs * np.linalg.norm(v - np.array(site))            # float64 geometry
        assert out[i]["status"] == 0
        assert abs(float(out[i]["dist"]) - d) <= 1e-6 * max(1.0, d)
        assert abs(float(out[i]["clearance"]) - (d - 0.05)) <= 2e-6
        centre = np.asarray(org) + (np.array(site) + 0.5) * vs
        assert np.allclose(out[i]["nearest"], centre, atol=1e-6)
        assert out[i]["idx"] == site[0] + dims[0] * (site[1] + dims[1] * site[2])


def test_query_occupied_outside_empty(oracle_mod):
    dims, vs, org = (8, 8, 8), 0.125, (0.0, 0.0, 0.0)
    occ = synth.sites_occupancy(dims, [(2, 3, 4)])
    sq, ix = oracle_mod.edt(occ)
    c = np.array([[2.5 * vs, 3.5 * vs, 4.5 * vs],     # on the occupied voxel
                  [1.0, 0.5, 0.5],                     # x = 8 voxels: upper face, outside
                  [-0.01, 0.5, 0.5]], dtype=np.float32)
    out = oracle_mod.query_spheres(sq, ix, dims, vs, org, c, np.full(3, 0.05, np.float32))
    assert out[0]["status"] == 0 and out[0]["dist"] == 0.0 and out[0]["sqdist"] == 0
    assert out[1]["status"] == 1 and np.isnan(out[1]["dist"]) and out[1]["idx"] == -1
    assert out[2]["status"] == 1
    e_sq, e_ix = oracle_mod.edt(np.zeros_like(occ))
    out = oracle_mod.query_spheres(e_sq, e_ix, dims, vs, org, c[:1], np.full(1, 0.05, np.float32))
    assert out[0]["status"] == 2 and np.isinf(out[0]["dist"]) and out[0]["idx"] == -1
