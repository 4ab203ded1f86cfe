"""Incremental EDT (vedt_map_set_incremental): a grid whose occupancy is unchanged since
its last EDT keeps its fields and skips all three passes; every recomputed field is
bit-exact against the oracle.  The static-scene reuse of Sec. IV: one EDT of a static
scene serves while the arm moves."""
import numpy as np
import pytest

import oracle
from paper_2407_02363_b300 import synth
from gpu_helpers import check_idx_valid, lib

pytestmark = pytest.mark.gpu


def field_np(m, which):
    sq, ix = m.field(which)
    return sq.cpu().numpy(), ix.cpu().numpy()


def assert_exact(m, which, occ):
    sq, ix = field_np(m, which)
    osq, _ = oracle.edt(occ)
    assert np.array_equal(sq, osq)
    check_idx_valid(occ, sq, ix)


@pytest.mark.parametrize("dims", [(96, 80, 72), (300, 20, 10)])
def test_unchanged_grids_are_skipped_and_changed_ones_recomputed(dims):
    v = lib()
    occ_e = synth.random_occupancy(3 + sum(dims), dims, 0.01)
    occ_s = synth.random_occupancy(4 + sum(dims), dims, 0.02)
    m = v.Map(dims, 0.01)
    m.set_incremental(True)
    m.upload_occupancy(v.MAP_ENV, occ_e)
    m.upload_occupancy(v.MAP_SELF, occ_s)
    m.compute_edt(v.MAP_BOTH)
    assert m.edt_recomputed(v.MAP_BOTH) == [True, True]
    assert_exact(m, v.MAP_ENV, occ_e)
    assert_exact(m, v.MAP_SELF, occ_s)

    # Nothing changed: both grids skipped.  Overwrite the fields to see that no pass ran.
    for g in (v.MAP_ENV, v.MAP_SELF):
        sq, _ = m.field_view(g)
        sq.fill_(-7)
    m.compute_edt(v.MAP_BOTH)
    assert m.edt_recomputed(v.MAP_BOTH) == [False, False]
    assert (field_np(m, v.MAP_ENV)[0] == -7).all() and (field_np(m, v.MAP_SELF)[0] == -7).all()

    # One voxel of the self grid flips: only the self grid is recomputed, exactly.
    occ_s2 = occ_s.copy()
    occ_s2[dims[2] // 2, dims[1] // 3, dims[0] - 1] ^= 1
    m.upload_occupancy(v.MAP_SELF, occ_s2)
    m.compute_edt(v.MAP_BOTH)
    assert m.edt_recomputed(v.MAP_BOTH) == [False, True]
    assert (field_np(m, v.MAP_ENV)[0] == -7).all()
    assert_exact(m, v.MAP_SELF, occ_s2)

    # A single-grid call only looks at its grid.
    occ_e2 = occ_e.copy()
    occ_e2[0, 0, 0] ^= 1
    m.upload_occupancy(v.MAP_ENV, occ_e2)
    m.compute_edt(v.MAP_ENV)
    assert m.edt_recomputed(v.MAP_ENV) == [True]
    assert_exact(m, v.MAP_ENV, occ_e2)

    # Switching incremental off recomputes every time.
    m.set_incremental(False)
    m.compute_edt(v.MAP_SELF)
    assert m.edt_recomputed(v.MAP_SELF) == [True]
    assert_exact(m, v.MAP_SELF, occ_s2)
    m.close()


def test_enabling_recomputes_even_if_the_snapshot_happens_to_match():
    """The first EDT after enabling never trusts fields it did not compute."""
    v = lib()
    dims = (40, 33, 21)
    occ = synth.random_occupancy(9, dims, 0.05)
    m = v.Map(dims, 0.01)
    m.upload_occupancy(v.MAP_ENV, occ)
    m.set_incremental(True)
    m.compute_edt(v.MAP_ENV)
    m.set_incremental(False)
    sq, _ = m.field_view(v.MAP_ENV)
    sq.fill_(-3)
    m.set_incremental(True)   # the snapshot still equals the occupancy
    m.compute_edt(v.MAP_ENV)
    assert m.edt_recomputed(v.MAP_ENV) == [True]
    assert_exact(m, v.MAP_ENV, occ)
    m.close()


def test_static_scene_with_moving_arm_reuses_the_environment_field():
    """Every frame clears both grids and reinserts the same static cloud and the moving
    arm: the environment EDT runs once, the self EDT every frame, all fields exact."""
    v = lib()
    grid = synth.GridSpec((64, 64, 64), 0.02)
    chain = synth.make_chain(11, (0.64, 0.64, 0.3))
    links = synth.link_models(chain, grid.voxel_size)
    cloud = synth.surface_cloud(12, grid, 20_000)
    import torch
    cloud_dev = torch.from_numpy(cloud).cuda()
    m = v.Map(grid.dims, grid.voxel_size, grid.origin)
    m.register_links(links)
    m.set_incremental(True)
    qs = synth.joint_trajectory(13, 4)
    for f, q in enumerate(qs):
        poses = oracle.fk(chain, q).astype(np.float32)
        m.clear(v.MAP_BOTH)
        m.insert_links(poses, 0b111)
        m.insert_pointcloud(cloud_dev, filter_self=False)
        m.compute_edt(v.MAP_BOTH)
        env_again, self_again = m.edt_recomputed(v.MAP_BOTH)
        assert env_again == (f == 0)
        e = np.zeros((64, 64, 64), np.uint8)
        s = np.zeros_like(e)
        oracle.insert_links(s, grid.dims, grid.voxel_size, grid.origin, links, poses, 0b111)
        oracle.insert_points(e, s, grid.dims, grid.voxel_size, grid.origin, cloud, filter_self=False)
        assert_exact(m, v.MAP_ENV, e)
        assert_exact(m, v.MAP_SELF, s)
        if f > 0:
            assert self_again == (not np.array_equal(s, prev_s))
        prev_s = s
    m.close()
