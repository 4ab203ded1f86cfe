"""GPU parity of batched maps (one persistent EDT launch over many grids of uneven
extents, batched insert/query launches, CUDA-graph replay) against the oracle and against
the same maps computed one at a time."""
import numpy as np
import pytest
import torch

import oracle
from paper_2407_02363_b300 import synth
from gpu_helpers import check_idx_valid, lib, spheres_bitequal

pytestmark = pytest.mark.gpu

SELF_MASK = 0b111


def _maps(v, dims_list, vs=0.02):
    return [v.Map(tuple(int(x) for x in d), vs) for d in dims_list]


@pytest.mark.parametrize("persistent,ctas,rows", [(1, 0, 32), (1, 1, 7), (1, 3, 128), (0, 0, 32)])
def test_batch_edt_uneven_maps(persistent, ctas, rows):
    v = lib()
    dims_list = synth.batch_dims(11, n_maps=10)
    maps = _maps(v, dims_list)
    occs = []
    for i, (m, d) in enumerate(zip(maps, dims_list)):
        e = synth.random_occupancy(100 + i, tuple(d), 0.003 * (1 + i % 3))
        s = synth.random_occupancy(200 + i, tuple(d), 0.0005) if i % 4 else np.zeros_like(e)
        m.upload_occupancy(v.MAP_ENV, e)
        m.upload_occupancy(v.MAP_SELF, s)
        occs.append((e, s))
    b = v.Batch(maps, stream=torch.cuda.Stream())
    b.set_tuning(ctas, rows, persistent)
    b.compute_edt()
    b.check()
    for m, (e, s) in zip(maps, occs):
        for g, occ in ((v.MAP_ENV, e), (v.MAP_SELF, s)):
            sq, ix = (t.cpu().numpy() for t in m.field(g))
            osq, _ = oracle.edt(occ)
            assert np.array_equal(sq, osq)
            check_idx_valid(occ, sq, ix)
    b.close()


def test_batch_mixed_small_and_large_matches_single_runs():
    v = lib()
    dims_list = [(64, 70, 90), (300, 40, 30), (128, 128, 20), (40, 20, 600)]
    maps = _maps(v, dims_list)
    occs = [synth.random_occupancy(7 + i, d, 0.004) for i, d in enumerate(dims_list)]
    for m, o in zip(maps, occs):
        m.upload_occupancy(v.MAP_ENV, o)
        m.upload_occupancy(v.MAP_SELF, o[::-1].copy())
    b = v.Batch(maps, stream=torch.cuda.Stream())
    b.compute_edt()
    b.check()
    batched = [tuple(t.cpu().numpy() for t in m.field(v.MAP_ENV)) for m in maps]
    for m, (sq, ix), o in zip(maps, batched, occs):
        m.compute_edt(v.MAP_ENV)         # alone, through the single-map path
        sq1, ix1 = (t.cpu().numpy() for t in m.field(v.MAP_ENV))
        assert np.array_equal(sq, sq1) and np.array_equal(ix, ix1)
        assert np.array_equal(sq, oracle.edt(o)[0])
    # both pass-Z tile shapes for the small grids (the large grids keep 32 x 1 rows), with
    # the persistent launch and with three plain launches
    for tz in (8, 32):
        b.set_tile_z(tz)
        assert b.tile_z() == tz
        for persistent in (1, 0):
            b.set_tuning(0, 32, persistent)
            for m in maps:
                m.field_view(v.MAP_ENV)[0].fill_(-5)
            torch.cuda.synchronize()
            b.compute_edt()
            b.check()
            for m, (sq, _) in zip(maps, batched):
                assert np.array_equal(m.field(v.MAP_ENV)[0].cpu().numpy(), sq), (tz, persistent)
    b.close()


def _frame_inputs(v, dims_list, chain, spheres, seed):
    """Config-3 style inputs: per map its own cloud (surface points scaled to the map's
    extent) and its own joint state; oracle FK poses and sphere centres."""
    clouds, poses, centres = [], [], []
    qs = synth.joint_states(seed, len(dims_list))
    for i, d in enumerate(dims_list):
        grid = synth.GridSpec(tuple(int(x) for x in d), 0.02)
        clouds.append(synth.surface_cloud(seed + i, grid, 50_000))
        ch = synth.Chain(base=chain.base.copy(), offsets=chain.offsets, lengths=chain.lengths, radius=chain.radius)
        ch.base[:, 3] = np.array(grid.extent) / 2
        poses.append(oracle.fk(ch, qs[i]).astype(np.float32))
        centres.append(oracle.sphere_centres(ch, spheres, qs[i]))
    offs = np.zeros(len(dims_list) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([len(c) for c in clouds])
    return clouds, offs, np.stack(poses), np.stack(centres)


def _oracle_frame(d, links, pose, cloud, centres, radii):
    X, Y, Z = (int(x) for x in d)
    s = np.zeros((Z, Y, X), np.uint8)
    oracle.insert_links(s, (X, Y, Z), 0.02, (0, 0, 0), links, pose, SELF_MASK)
    e = np.zeros_like(s)
    oracle.insert_points(e, s, (X, Y, Z), 0.02, (0, 0, 0), cloud, filter_self=True)
    return e, s


def test_batch_pipeline_and_graph_replay():
    v = lib()
    dims_list = synth.batch_dims(1234 + 3000, n_maps=12)
    chain = synth.make_chain(1234 + 3000, (0.0, 0.0, 0.0))
    links = synth.link_models(chain, 0.02)
    spheres = synth.sphere_model(chain)
    m_sph = len(spheres.radius)
    maps = _maps(v, dims_list)
    stream = torch.cuda.Stream()
    b = v.Batch(maps, stream=stream)
    b.register_links(links)
    radii = torch.from_numpy(spheres.radius).cuda()
    for frame, seed in enumerate((1, 2, 3)):
        clouds, offs, poses, centres = _frame_inputs(v, dims_list, chain, spheres, 1234 + 3000 + 10 * seed)
        if frame == 0:
            cap = int(max(offs[1:] - offs[:-1]))
            xyz = torch.zeros((int(offs[-1]) + 1024, 3), dtype=torch.float32, device="cuda")
            cen = torch.zeros((len(maps), m_sph, 3), dtype=torch.float32, device="cuda")
            out = torch.zeros(len(maps) * 2 * m_sph * 32, dtype=torch.uint8, device="cuda")
        xyz[: offs[-1]] = torch.from_numpy(np.concatenate(clouds)).cuda()
        cen.copy_(torch.from_numpy(centres).cuda())
        torch.cuda.synchronize()
        b.set_frame(xyz, offs, poses, SELF_MASK, cen, radii, m_sph, out)
        if frame == 0:
            b.run()
        elif frame == 1:
            b.capture()
            b.replay()
        else:
            b.replay()
        b.check()
        res = out.cpu().numpy().view(v.SPHERE_DTYPE).reshape(len(maps), 2, m_sph)
        for i, (m, d) in enumerate(zip(maps, dims_list)):
            e, s = _oracle_frame(d, links, poses[i], clouds[i], centres[i], spheres.radius)
            assert np.array_equal(m.occupancy(v.MAP_ENV).cpu().numpy(), e)
            assert np.array_equal(m.occupancy(v.MAP_SELF).cpu().numpy(), s)
            for g, occ in ((0, e), (1, s)):
                sq, ix = (t.cpu().numpy() for t in m.field(v.MAP_ENV if g == 0 else v.MAP_SELF))
                osq, _ = oracle.edt(occ)
                assert np.array_equal(sq, osq)
                exp = oracle.query_spheres(osq, ix, tuple(int(x) for x in d), 0.02, (0, 0, 0), centres[i],
                                           spheres.radius)
                got = res[i, g].copy()
                e2 = np.zeros(m_sph, dtype=got.dtype)
                for name in e2.dtype.names:
                    e2[name] = exp[name]
                assert spheres_bitequal(got, e2)
        if frame == 0:
            assert cap > 0
    b.close()
