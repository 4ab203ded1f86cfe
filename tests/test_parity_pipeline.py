"""GPU parity of the whole per-frame pipeline (Alg. 2 lines 4-10) against the oracle:
occupancy after ClearMap + Insert(O_Lk) + Insert(Point_Cloud) byte-equal, EDT of both
maps bit-exact in squared distance, sphere results (Eq. (dist)) bit-equal."""
import numpy as np
import pytest
import torch

import oracle
from paper_2407_02363_b300 import synth
from gpu_helpers import check_idx_valid, lib, spheres_bitequal

pytestmark = pytest.mark.gpu

SELF_MASK = 0b111   # static body + links 1-2 form the self-collision obstacle O_L


def robot_points(link_models, poses, mask, n, seed):
    """Cloud points lying on the robot (to exercise the robot-point removal)."""
    rng = np.random.default_rng(seed)
    pts = []
    for k, P in enumerate(poses):
        if not (mask >> k) & 1 or len(link_models[k]) == 0:
            continue
        sel = link_models[k][rng.integers(0, len(link_models[k]), n)].astype(np.float64)
        pts.append(sel @ P[:, :3].T.astype(np.float64) + P[:, 3])
    return np.concatenate(pts).astype(np.float32)


def run_frame(grid, chain, q, cloud, T=None, use_library_fk=False):
    v = lib()
    links = synth.link_models(chain, grid.voxel_size)
    spheres = synth.sphere_model(chain)
    poses = oracle.fk(chain, q).astype(np.float32)
    m = v.Map(grid.dims, grid.voxel_size, grid.origin)
    m.register_links(links)
    m.clear(v.MAP_BOTH)
    if use_library_fk:
        m.insert_robot(chain, q, SELF_MASK)
    else:
        m.insert_links(poses, SELF_MASK)
    cl = torch.from_numpy(cloud).cuda()
    counts = torch.zeros(3, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    m.insert_pointcloud(cl, T_world_sensor=T, filter_self=True, counts_dev=counts)
    occ_env = m.occupancy(v.MAP_ENV).cpu().numpy()
    occ_self = m.occupancy(v.MAP_SELF).cpu().numpy()
    m.compute_edt(v.MAP_BOTH)
    fields = [tuple(t.cpu().numpy() for t in m.field(g)) for g in (v.MAP_ENV, v.MAP_SELF)]
    centres = oracle.sphere_centres(chain, spheres, q)
    res = m.query_spheres(centres, spheres.radius, v.MAP_BOTH)
    m.close()
    # oracle
    X, Y, Z = grid.dims
    o_self = np.zeros((Z, Y, X), np.uint8)
    oracle.insert_links(o_self, grid.dims, grid.voxel_size, grid.origin, links, poses, SELF_MASK)
    o_env = np.zeros((Z, Y, X), np.uint8)
    n_written = oracle.insert_points(o_env, o_self, grid.dims, grid.voxel_size, grid.origin, cloud, T=T,
                                     filter_self=True)
    return dict(occ_env=occ_env, occ_self=occ_self, o_env=o_env, o_self=o_self, fields=fields,
                res=res, centres=centres, radii=spheres.radius, counts=counts.cpu().numpy(),
                n_written=n_written, n_points=len(cloud))


def check_frame(grid, r):
    assert np.array_equal(r["occ_self"], r["o_self"])
    assert np.array_equal(r["occ_env"], r["o_env"])
    assert r["counts"][0] == r["n_written"] and r["counts"].sum() == r["n_points"]
    m = len(r["radii"])
    for g, occ in enumerate((r["o_env"], r["o_self"])):
        sq, ix = r["fields"][g]
        osq, oix = oracle.edt(occ)
        assert np.array_equal(sq, osq)
        check_idx_valid(occ, sq, ix)
        # the query reads the oracle's own field so ties in idx cannot matter
        expect = oracle.query_spheres(osq, ix, grid.dims, grid.voxel_size, grid.origin, r["centres"], r["radii"])
        got = r["res"][g * m:(g + 1) * m].copy()
        exp = np.zeros(m, dtype=got.dtype)
        for name in exp.dtype.names:
            exp[name] = expect[name]
        assert spheres_bitequal(got, exp)
        # and against the oracle's own idx, everything but idx/nearest must agree too
        e2 = oracle.query_spheres(osq, oix, grid.dims, grid.voxel_size, grid.origin, r["centres"], r["radii"])
        for name in ("sqdist", "status"):
            assert np.array_equal(got[name], e2[name])
        assert np.array_equal(got["dist"].view(np.uint32), e2["dist"].view(np.uint32))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_config1_frame(seed):
    """64^3 at 2 cm: 20k surface points + robot points, 7-DoF capsule chain, 24 spheres."""
    grid = synth.GridSpec((64, 64, 64), 0.02)
    chain = synth.make_chain(1234 + 1000 + seed, (0.64, 0.64, 0.64))
    q = synth.joint_states(1234 + 1000 + seed, 1)[0]
    cloud = synth.surface_cloud(1234 + 1000 + seed, grid, 20_000)
    poses = oracle.fk(chain, q).astype(np.float32)
    extra = robot_points(synth.link_models(chain, grid.voxel_size), poses, SELF_MASK, 500, seed)
    cloud = np.concatenate([cloud, extra, np.array([[np.nan, 0, 0], [9, 9, 9]], np.float32)])
    r = run_frame(grid, chain, q, cloud)
    assert r["counts"][2] > 0            # some robot points were removed
    check_frame(grid, r)


def test_config1_library_fk_and_sensor_pose():
    grid = synth.GridSpec((64, 64, 64), 0.02, origin=(-0.64, -0.64, 0.0))
    chain = synth.make_chain(77, (0.0, 0.0, 0.64))
    q = synth.joint_states(78, 1)[0]
    cloud = synth.surface_cloud(79, synth.GridSpec((64, 64, 64), 0.02), 20_000)
    T = np.array([[0, -1, 0, 0.3], [1, 0, 0, -0.9], [0, 0, 1, 0.01]], dtype=np.float32)
    r = run_frame(grid, chain, q, cloud, T=T, use_library_fk=True)
    check_frame(grid, r)


def test_config2_frame_full_size():
    """256^3 at 1 cm: 300k-point depth-camera cloud with the moving sphere obstacle."""
    grid = synth.GridSpec((256, 256, 256), 0.01)
    scene = synth.CameraScene(1234 + 2000, grid)
    chain = synth.make_chain(1234 + 2000, (1.28, 1.28, 1.28))
    q = synth.joint_trajectory(1234 + 2000, 40)[37]
    cloud = scene.frame(37)
    r = run_frame(grid, chain, q, cloud)
    assert r["occ_env"].mean() > 0.001
    check_frame(grid, r)


@pytest.mark.parametrize("timing", [False, True])
def test_frame_api_full_size_on_two_streams(timing):
    """vedt_frame, the call the bench times: the self map's EDT on the side stream, the
    cloud and the environment EDT on the map's stream, then the query; several frames
    back to back.  Each frame's fields and sphere results against the oracle (with
    per-kernel timing on, the same launches run serially)."""
    v = lib()
    grid = synth.GridSpec((256, 256, 256), 0.01)
    scene = synth.CameraScene(1234 + 2000, grid)
    chain = synth.make_chain(1234 + 2000, (1.28, 1.28, 1.28))
    links = synth.link_models(chain, grid.voxel_size)
    spheres = synth.sphere_model(chain)
    traj = synth.joint_trajectory(1234 + 2000, 40)
    m = v.Map(grid.dims, grid.voxel_size, grid.origin, stream=torch.cuda.Stream())
    m.register_links(links)
    m.set_timing(timing)
    cchain = v.make_chain(chain)
    nm = len(spheres.radius)
    out = torch.empty(2 * nm * 32, dtype=torch.uint8, device="cuda")
    radii = torch.from_numpy(spheres.radius).cuda()
    for f in (30, 31, 32):
        cloud = scene.frame(f)
        cl = torch.from_numpy(cloud).cuda()
        centres_np = oracle.sphere_centres(chain, spheres, traj[f])
        centres = torch.from_numpy(centres_np).cuda()
        torch.cuda.synchronize()
        m.frame(cl, cl.shape[0], cchain, traj[f], SELF_MASK, centres, radii, nm, out)
        m.check()
        res = out.cpu().numpy().view(v.SPHERE_DTYPE)
        poses = v.fk(chain, traj[f]).astype(np.float32)
        X, Y, Z = grid.dims
        o_self = np.zeros((Z, Y, X), np.uint8)
        oracle.insert_links(o_self, grid.dims, grid.voxel_size, grid.origin, links, poses, SELF_MASK)
        o_env = np.zeros((Z, Y, X), np.uint8)
        oracle.insert_points(o_env, o_self, grid.dims, grid.voxel_size, grid.origin, cloud, filter_self=True)
        for g, occ in ((v.MAP_ENV, o_env), (v.MAP_SELF, o_self)):
            sq, ix = (t.cpu().numpy() for t in m.field(g))
            osq, _ = oracle.edt(occ)
            assert np.array_equal(sq, osq)
            check_idx_valid(occ, sq, ix)
            k = 0 if g == v.MAP_ENV else 1
            expect = oracle.query_spheres(osq, ix, grid.dims, grid.voxel_size, grid.origin, centres_np,
                                          spheres.radius)
            got = res[k * nm:(k + 1) * nm].copy()
            exp = np.zeros(nm, dtype=got.dtype)
            for name in exp.dtype.names:
                exp[name] = expect[name]
            assert spheres_bitequal(got, exp)
    m.close()


def test_frame_api_back_to_back_without_host_syncs():
    """Frames queued back to back on the map's stream, as the bench times them: no host
    synchronisation between frames, so each frame's first kernel is launched while the
    previous frame's query still runs (and waits for it).  Every frame writes its sphere
    results to a buffer of its own; each frame's results, and the last frame's fields,
    against the oracle."""
    v = lib()
    grid = synth.GridSpec((256, 256, 256), 0.01)
    scene = synth.CameraScene(1234 + 2000, grid)
    chain = synth.make_chain(1234 + 2000, (1.28, 1.28, 1.28))
    links = synth.link_models(chain, grid.voxel_size)
    spheres = synth.sphere_model(chain)
    traj = synth.joint_trajectory(1234 + 2000, 40)
    m = v.Map(grid.dims, grid.voxel_size, grid.origin, stream=torch.cuda.Stream())
    m.register_links(links)
    cchain = v.make_chain(chain)
    nm = len(spheres.radius)
    radii = torch.from_numpy(spheres.radius).cuda()
    frames = (20, 21, 22, 23)
    clouds = {f: scene.frame(f) for f in frames}
    cl = {f: torch.from_numpy(clouds[f]).cuda() for f in frames}
    cen_np = {f: oracle.sphere_centres(chain, spheres, traj[f]) for f in frames}
    cen = {f: torch.from_numpy(cen_np[f]).cuda() for f in frames}
    outs = {f: torch.empty(2 * nm * 32, dtype=torch.uint8, device="cuda") for f in frames}
    torch.cuda.synchronize()
    for f in frames:
        m.frame(cl[f], cl[f].shape[0], cchain, traj[f], SELF_MASK, cen[f], radii, nm, outs[f])
    m.check()
    X, Y, Z = grid.dims
    for f in frames:
        poses = v.fk(chain, traj[f]).astype(np.float32)
        o_self = np.zeros((Z, Y, X), np.uint8)
        oracle.insert_links(o_self, grid.dims, grid.voxel_size, grid.origin, links, poses, SELF_MASK)
        o_env = np.zeros((Z, Y, X), np.uint8)
        oracle.insert_points(o_env, o_self, grid.dims, grid.voxel_size, grid.origin, clouds[f], filter_self=True)
        res = outs[f].cpu().numpy().view(v.SPHERE_DTYPE)
        for k, (g, occ) in enumerate(((v.MAP_ENV, o_env), (v.MAP_SELF, o_self))):
            osq, oix = oracle.edt(occ)
            if f == frames[-1]:
                sq, ix = (t.cpu().numpy() for t in m.field(g))
                assert np.array_equal(sq, osq)
                check_idx_valid(occ, sq, ix)
            expect = oracle.query_spheres(osq, oix, grid.dims, grid.voxel_size, grid.origin, cen_np[f],
                                          spheres.radius)
            got = res[k * nm:(k + 1) * nm].copy()
            exp = np.zeros(nm, dtype=got.dtype)
            for name in exp.dtype.names:
                exp[name] = expect[name]
            # the nearest voxel may be any occupied voxel at that distance: compare what is
            # unique bit for bit, and check that the returned voxel is one of them
            assert np.array_equal(got["sqdist"], exp["sqdist"]) and np.array_equal(got["status"], exp["status"])
            for name in ("dist", "clearance"):
                assert np.array_equal(got[name].view(np.uint32), exp[name].view(np.uint32)), (f, name)
            vox = np.floor((cen_np[f].astype(np.float32) - np.asarray(grid.origin, np.float32))
                           / np.float32(grid.voxel_size)).astype(np.int64)
            for i in np.nonzero(got["status"] == v.SPHERE_OK)[0]:
                j = int(got["idx"][i])
                nx, ny, nz = j % X, (j // X) % Y, j // (X * Y)
                assert occ[nz, ny, nx] != 0
                assert (nx - vox[i, 0]) ** 2 + (ny - vox[i, 1]) ** 2 + (nz - vox[i, 2]) ** 2 == got["sqdist"][i]
    m.close()


def test_async_host_frames_back_to_back_match_sync_frames():
    """Frames queued back to back with vedt_frame_host_async alternate the two staging
    buffers, each upload running on the copy stream while the previous frame computes;
    frame by frame they give the results of the synchronous call on the same inputs.  A
    larger cloud midway grows the staging buffers while frames are in flight.  The
    asynchronous frames' outputs are page-locked (the query kernel writes them directly),
    the synchronous frames' are numpy arrays (copied after the frame)."""
    v = lib()
    grid = synth.GridSpec((96, 96, 96), 0.02)
    chain = synth.make_chain(4321, (0.96, 0.96, 0.96))
    links = synth.link_models(chain, grid.voxel_size)
    spheres = synth.sphere_model(chain)
    cc = v.make_chain(chain)
    frames = []
    for i in range(6):
        cloud = synth.surface_cloud(500 + i, grid, 20_000 if i < 3 else 60_000)
        q = synth.joint_states(600 + i, 1)[0]
        cen = oracle.sphere_centres(chain, spheres, q).astype(np.float32)
        frames.append((torch.from_numpy(cloud).pin_memory(), q, cen))
    ref_map = v.Map(grid.dims, grid.voxel_size, grid.origin)
    ref_map.register_links(links)
    refs = [ref_map.frame_host(c.numpy(), cc, q, SELF_MASK, cen, spheres.radius) for c, q, cen in frames]
    m = v.Map(grid.dims, grid.voxel_size, grid.origin)
    m.register_links(links)
    item = v.SPHERE_DTYPE.itemsize
    outs = [torch.zeros(2 * len(spheres.radius) * item, dtype=torch.uint8).pin_memory() for _ in frames]
    for (c, q, cen), o in zip(frames, outs):
        m.frame_host_async(c, cc, q, SELF_MASK, cen, spheres.radius, o)
    while not m.done():
        pass
    for ref, o in zip(refs, outs):
        assert spheres_bitequal(o.numpy().view(v.SPHERE_DTYPE), ref)
    # the synchronous call after asynchronous ones still agrees
    again = m.frame_host(frames[0][0].numpy(), cc, frames[0][1], SELF_MASK, frames[0][2], spheres.radius)
    assert spheres_bitequal(again, refs[0])
    m.close()
    ref_map.close()


def test_empty_cloud_and_all_outside():
    v = lib()
    grid = synth.GridSpec((32, 32, 32), 0.05)
    m = v.Map(grid.dims, grid.voxel_size)
    m.clear(v.MAP_BOTH)
    m.insert_pointcloud(torch.zeros((0, 3), device="cuda"), n=0)
    far = torch.full((100, 3), 50.0, device="cuda")
    counts = torch.zeros(3, dtype=torch.int64, device="cuda")
    m.insert_pointcloud(far, counts_dev=counts)
    m.compute_edt(v.MAP_BOTH)
    res = m.query_spheres(np.array([[0.5, 0.5, 0.5], [5, 5, 5]], np.float32), np.array([0.05, 0.05], np.float32))
    assert counts.cpu().tolist() == [0, 100, 0]
    assert res["status"].tolist() == [v.SPHERE_EMPTY, v.SPHERE_OUTSIDE] * 2
    assert np.isinf(res["dist"][0]) and np.isnan(res["dist"][1])
    m.close()


def test_timing_api_counts_launches():
    v = lib()
    m = v.Map((64, 64, 64), 0.02)
    m.set_timing(True)
    for _ in range(3):
        m.clear(v.MAP_BOTH)
        m.compute_edt(v.MAP_BOTH)
    t = m.kernel_times()
    # ClearMap of both grids is one launch (the two grids share one allocation)
    assert t["edt_x"][1] == 3 and t["edt_y"][1] == 3 and t["edt_z"][1] == 3 and t["clear"][1] == 3
    assert all(ms >= 0 for ms, _ in t.values())
    m.close()


def test_bounded_wait_expires_with_status_not_hang():
    """A wait on a counter nothing sets gives up after its limit, flags the error word,
    and the host reads ETIMEOUT; the context keeps working afterwards."""
    v = lib()
    s = torch.cuda.Stream()
    assert v._lib.vedt_selftest_wait(s.cuda_stream, 1 << 12) == v.ETIMEOUT
    m = v.Map((16, 16, 16), 0.1)
    m.compute_edt(v.MAP_BOTH)
    m.check()
    m.close()
