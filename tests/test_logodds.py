"""GPU parity of the Bayesian (log-odds) occupancy of the environment map (Sec. III-A)
against the oracle chain: frame after frame, the occupancy the EDT sees and its field are
byte- and bit-equal to oracle.logodds.update applied to the oracle's insertion."""
import numpy as np
import pytest
import torch

import oracle
from oracle import logodds
from paper_2407_02363_b300 import synth
from gpu_helpers import check_idx_valid, lib

pytestmark = pytest.mark.gpu

SELF_MASK = 0b111
PARAMS = dict(l_hit=9, l_miss=4, l_min=-20, l_max=40, threshold=15)


def occ_np(m, which):
    return m.occupancy(which).cpu().numpy()


def run_steps(dims, frames, params, seed):
    """Step API: upload each frame's hits into M_I, update, compare occupancy with the
    oracle chain; returns the per-frame occupancies."""
    v = lib()
    m = v.Map(dims, 0.01)
    m.set_logodds(True, **params)
    X, Y, Z = dims
    L = np.zeros((Z, Y, X), np.int8)
    got = []
    for f in range(frames):
        hit = synth.random_occupancy(seed + f, dims, 0.3 if f % 3 else 0.05)
        m.upload_occupancy(v.MAP_ENV, hit)
        m.update_occupancy()
        L, occ = logodds.update(L, hit, **params)
        g = occ_np(m, v.MAP_ENV)
        assert np.array_equal(g, occ), f"frame {f}: {int((g != occ).sum())} voxels differ"
        got.append(g)
    m.close()
    return got


@pytest.mark.parametrize("dims", [(40, 30, 20), (33, 7, 5), (1, 1, 1), (300, 17, 3)])
def test_step_api_matches_oracle_chain(dims):
    run_steps(dims, 12, PARAMS, 100 + sum(dims))


@pytest.mark.parametrize("params", [
    dict(l_hit=255, l_miss=255, l_min=-128, l_max=127, threshold=1),     # saturating steps
    dict(l_hit=1, l_miss=0, l_min=0, l_max=3, threshold=3),              # never forgets
    dict(l_hit=0, l_miss=7, l_min=-30, l_max=0, threshold=-10),          # occupied until missed twice
    dict(l_hit=5, l_miss=1, l_min=-5, l_max=20, threshold=127),          # threshold above l_max: empty
])
def test_clamps_and_degenerate_parameters(params):
    got = run_steps((24, 20, 18), 10, params, 7)
    if params["threshold"] > params["l_max"]:
        assert all(g.sum() == 0 for g in got)


def test_reduces_to_one_hit_rule():
    """l_min = 0, l_miss = l_max and 0 < l_hit = threshold <= l_max: the occupancy is
    this frame's hits."""
    v = lib()
    dims = (50, 40, 30)
    m = v.Map(dims, 0.01)
    m.set_logodds(True, l_hit=6, l_miss=30, l_min=0, l_max=30, threshold=6)
    for f in range(6):
        hit = synth.random_occupancy(f, dims, 0.2)
        m.upload_occupancy(v.MAP_ENV, hit)
        m.update_occupancy()
        assert np.array_equal(occ_np(m, v.MAP_ENV), hit)
    m.close()


@pytest.mark.parametrize("timing", [False, True])
def test_frame_api_sequence_with_logodds(timing):
    """vedt_frame with the log-odds update between the insertion and the EDT: a moving
    camera scene whose occupancy lags the hits (a voxel needs two hits, and fades after
    some misses); M_I occupancy, both fields and their indices against the oracle."""
    v = lib()
    grid = synth.GridSpec((128, 128, 128), 0.02)
    scene = synth.CameraScene(4321, grid, n_points=60_000)
    chain = synth.make_chain(4321, (1.28, 1.28, 1.28))
    links = synth.link_models(chain, grid.voxel_size)
    spheres = synth.sphere_model(chain)
    traj = synth.joint_trajectory(4321, 20)
    m = v.Map(grid.dims, grid.voxel_size, grid.origin, stream=torch.cuda.Stream())
    m.register_links(links)
    m.set_timing(timing)
    m.set_logodds(True, **PARAMS)
    cchain = v.make_chain(chain)
    nm = len(spheres.radius)
    out = torch.empty(2 * nm * 32, dtype=torch.uint8, device="cuda")
    radii = torch.from_numpy(spheres.radius).cuda()
    X, Y, Z = grid.dims
    L = np.zeros((Z, Y, X), np.int8)
    lag = 0
    for f in range(6):
        cloud = scene.frame(10 + 3 * f)
        cl = torch.from_numpy(cloud).cuda()
        centres = torch.from_numpy(oracle.sphere_centres(chain, spheres, traj[f])).cuda()
        torch.cuda.synchronize()
        m.frame(cl, cl.shape[0], cchain, traj[f], SELF_MASK, centres, radii, nm, out)
        m.check()
        poses = v.fk(chain, traj[f]).astype(np.float32)
        o_self = np.zeros((Z, Y, X), np.uint8)
        oracle.insert_links(o_self, grid.dims, grid.voxel_size, grid.origin, links, poses, SELF_MASK)
        hit = np.zeros((Z, Y, X), np.uint8)
        oracle.insert_points(hit, o_self, grid.dims, grid.voxel_size, grid.origin, cloud, filter_self=True)
        L, o_env = logodds.update(L, hit, **PARAMS)
        lag += int((o_env != hit).sum())
        assert np.array_equal(occ_np(m, v.MAP_ENV), o_env)
        for g, occ in ((v.MAP_ENV, o_env), (v.MAP_SELF, o_self)):
            sq, ix = (t.cpu().numpy() for t in m.field(g))
            osq, _ = oracle.edt(occ)
            assert np.array_equal(sq, osq)
            check_idx_valid(occ, sq, ix)
    assert lag > 0        # the filtered map differs from the one-hit map
    if timing:
        t = m.kernel_times()
        assert t["occupancy"][1] == 6 and t["insert_points"][1] == 6
    m.close()


def test_static_scene_settles_and_incremental_edt_skips():
    """A static cloud: once every voxel's log-odds has saturated, the occupancy stops
    changing and the incremental EDT skips the environment grid."""
    v = lib()
    dims = (64, 64, 64)
    m = v.Map(dims, 0.02)
    m.set_logodds(True, l_hit=10, l_miss=10, l_min=-20, l_max=20, threshold=15)
    m.set_incremental(True)
    hit = synth.random_occupancy(3, dims, 0.02)
    seen = []
    for f in range(5):
        m.upload_occupancy(v.MAP_ENV, hit)
        m.update_occupancy()
        m.compute_edt(v.MAP_ENV)
        seen.append(m.edt_recomputed(v.MAP_ENV)[0])
    # frame 0: all unknown -> nothing occupied yet (L = 10 < 15) but the first EDT runs;
    # frame 1: hits reach 20 -> occupied; later frames: saturated, nothing changes
    assert seen == [True, True, False, False, False]
    assert np.array_equal(occ_np(m, v.MAP_ENV), hit)
    sq, _ = m.field(v.MAP_ENV)
    assert np.array_equal(sq.cpu().numpy(), oracle.edt(hit)[0])
    m.close()


def test_turning_off_and_bad_arguments():
    v = lib()
    m = v.Map((16, 16, 16), 0.01)
    with pytest.raises(v.VedtError):
        m.update_occupancy()                         # off
    for bad in (dict(l_hit=-1), dict(l_miss=256), dict(l_min=1), dict(l_max=128), dict(l_min=-129),
                dict(threshold=-20)):
        p = dict(PARAMS, **bad)
        with pytest.raises(v.VedtError):
            m.set_logodds(True, **p)
    m.set_logodds(True, **PARAMS)
    hit = synth.random_occupancy(1, (16, 16, 16), 0.5)
    m.upload_occupancy(v.MAP_ENV, hit)
    m.update_occupancy()
    m.set_logodds(False)
    with pytest.raises(v.VedtError):
        m.update_occupancy()
    m.set_logodds(True, **PARAMS)                    # restarts from unknown
    m.upload_occupancy(v.MAP_ENV, hit)
    m.update_occupancy()
    assert occ_np(m, v.MAP_ENV).sum() == 0           # one hit (9) is below the threshold
    m.close()


@pytest.mark.parametrize("dims,incremental", [((300, 48, 40), False), ((96, 80, 72), True)])
def test_frames_on_the_standalone_update_path(dims, incremental):
    """Frames whose log-odds update cannot ride in pass X: a grid wider than 256 voxels,
    and an incremental map (its snapshot diff must see the updated occupancy).  No arm:
    the cloud alone, M_I against the oracle chain and its field exact."""
    v = lib()
    grid = synth.GridSpec(dims, 0.02)
    m = v.Map(grid.dims, grid.voxel_size, grid.origin, stream=torch.cuda.Stream())
    m.set_logodds(True, **PARAMS)
    m.set_incremental(incremental)
    X, Y, Z = dims
    L = np.zeros((Z, Y, X), np.int8)
    empty = np.zeros((Z, Y, X), np.uint8)
    for f in range(5):
        cloud = synth.surface_cloud(70 + (f % 3), grid, 30_000)      # frames 3 and 4 repeat 0 and 1
        cl = torch.from_numpy(cloud).cuda()
        torch.cuda.synchronize()
        m.frame(cl, cl.shape[0], None, None, 0, None, None, 0, None)
        m.check()
        hit = np.zeros((Z, Y, X), np.uint8)
        oracle.insert_points(hit, empty, grid.dims, grid.voxel_size, grid.origin, cloud, filter_self=True)
        L, occ = logodds.update(L, hit, **PARAMS)
        assert np.array_equal(occ_np(m, v.MAP_ENV), occ), f"frame {f}"
        sq, ix = (t.cpu().numpy() for t in m.field(v.MAP_ENV))
        assert np.array_equal(sq, oracle.edt(occ)[0])
        check_idx_valid(occ, sq, ix)
    m.close()
