"""Autotuner: cache keys, candidate sets, winner selection and cache round trip on the
CPU; on the GPU, real sweeps over a batch (launch shapes x band counts x pass-Z tile
shapes) and over a single map's band counts and tile shapes, with the fields equal to the
oracle at every candidate."""
import numpy as np
import pytest

from paper_2407_02363_b300 import autotune, synth


def test_signature_is_order_independent_and_kind_specific():
    a = autotune.signature("B300", [(64, 80, 90), (100, 100, 100)])
    b = autotune.signature("B300", [(100, 100, 100), (64, 80, 90)])
    c = autotune.signature("B300", [(100, 100, 100), (64, 80, 91)])
    d = autotune.signature("H100", [(100, 100, 100), (64, 80, 90)])
    e = autotune.signature("B300", [(64, 80, 90), (100, 100, 100)], kind="frame")
    assert a == b and a != c and a != d and a != e


def test_candidates_cover_bands_and_shapes():
    small = autotune.batch_candidates()
    assert {t[3] for t in small} == {1, 2, 4, 8}
    assert {t[4] for t in small} == {8, 32}
    assert any(t[0] == 0 for t in small) and any(t[0] == 1 for t in small)
    # every (launch shape, bands) pair at both tile shapes
    assert {t[:4] for t in small if t[4] == 8} == {t[:4] for t in small if t[4] == 32}
    assert {t[3] for t in autotune.batch_candidates(large=True)} == {0, 4, 8}
    assert autotune.map_candidates((256, 256, 256)) == (1, 2, 4, 8)
    assert autotune.map_candidates((512, 512, 128)) == (0, 4, 8)
    mt = autotune.map_tunings((256, 256, 256))
    assert set(mt) == {autotune.MapTuning(b, z) for b in (1, 2, 4, 8) for z in (8, 32)}
    assert set(autotune.map_tunings((512, 512, 128))) == {autotune.MapTuning(b, z) for b in (0, 4, 8) for z in (8, 32)}


def test_pick_smallest_and_cache_roundtrip(tmp_path):
    t1, t2, t3 = autotune.Tuning(1, 0, 32, 4), autotune.Tuning(1, 4, 8, 2), autotune.Tuning(0, 0, 32, 8)
    assert autotune.pick({t1: 2.0, t2: 1.5, t3: 3.0}) == t2
    assert autotune.pick({1: 0.3, 4: 0.2, 8: 0.25}) == 4
    p = str(tmp_path / "c.json")
    autotune.store_cache({"k": {"tuning": {"persistent": 1, "ctas_per_sm": 4, "rows_per_item": 8, "bands": 2,
                                           "tile_z": 32}}}, p)
    assert autotune.Tuning(**autotune.load_cache(p)["k"]["tuning"]) == autotune.Tuning(1, 4, 8, 2, 32)
    assert autotune.load_cache(str(tmp_path / "missing.json")) == {}
    # map entries: the current form and one written before tile shapes were tuned
    assert autotune._map_entry({"tuning": {"bands": 8, "tile_z": 32}}) == autotune.MapTuning(8, 32)
    assert autotune._map_entry({"bands": 2}) == autotune.MapTuning(2, 0)


def _batch_maps(v, seed, n, density):
    dims_list = synth.batch_dims(seed, n_maps=n)
    maps, occs = [], []
    for i, d in enumerate(dims_list):
        m = v.Map(tuple(int(x) for x in d), 0.02)
        o = synth.random_occupancy(seed + i, tuple(int(x) for x in d), density)
        s = synth.random_occupancy(seed + 100 + i, tuple(int(x) for x in d), density / 10)
        m.upload_occupancy(v.MAP_ENV, o)
        m.upload_occupancy(v.MAP_SELF, s)
        maps.append(m)
        occs.append((o, s))
    return dims_list, maps, occs


@pytest.mark.gpu
def test_tune_batch_sweeps_and_every_candidate_is_exact(tmp_path):
    import torch

    import oracle
    from gpu_helpers import lib
    v = lib()
    dims_list, maps, occs = _batch_maps(v, 5, 6, 0.002)
    ref = [(oracle.edt(o)[0], oracle.edt(s)[0]) for o, s in occs]
    st = torch.cuda.Stream()
    b = v.Batch(maps, stream=st)
    cands = [(0, 0, 32, 1, 8), (0, 0, 32, 8, 32), (1, 0, 32, 4, 8), (1, 2, 8, 2, 32), (1, 0, 64, 8, 8),
             (1, 4, 16, 1, 32), (0, 0, 32, 4, 0)]
    for c in cands:   # every candidate gives the oracle's fields
        for m in maps:
            for w in (v.MAP_ENV, v.MAP_SELF):
                m.field_view(w)[0].fill_(-5)
        torch.cuda.synchronize()   # the fills run on torch's stream, the batch on its own
        autotune.Tuning(*c).apply(b)
        b.compute_edt()
        b.check()
        for m, (re, rs) in zip(maps, ref):
            assert np.array_equal(m.field(v.MAP_ENV)[0].cpu().numpy(), re), c
            assert np.array_equal(m.field(v.MAP_SELF)[0].cpu().numpy(), rs), c
    path = str(tmp_path / "tune.json")
    best, times = autotune.tune(b, st, dims_list, candidates=cands, reps=2, path=path)
    assert len(times) == len(cands) and best in times and all(t > 0 for t in times.values())
    again, t2 = autotune.tune(b, st, dims_list, candidates=cands, path=path)
    assert again == best and t2 == {}           # served from the cache
    assert autotune.apply_cached(b, dims_list, path=path) == best
    b.close()
    for m in maps:
        m.close()


@pytest.mark.gpu
def test_tune_map_bands_exact_at_every_count(tmp_path):
    import torch

    import oracle
    from gpu_helpers import lib
    v = lib()
    dims = (96, 70, 130)
    o = synth.random_occupancy(3, dims, 0.003)
    st = torch.cuda.Stream()
    m = v.Map(dims, 0.02, stream=st)
    m.upload_occupancy(v.MAP_ENV, o)
    m.upload_occupancy(v.MAP_SELF, o)
    ref = oracle.edt(o)[0]
    path = str(tmp_path / "tune.json")
    best, times = autotune.tune_map(m, st, dims, reps=2, path=path)
    assert set(times) == set(autotune.map_tunings(dims)) and best in times
    assert m.tile_z() == best.tile_z
    for t in autotune.map_tunings(dims):
        t.apply(m)
        assert m.tile_z() == t.tile_z
        m.field_view(v.MAP_ENV)[0].fill_(-5)
        torch.cuda.synchronize()
        m.compute_edt(v.MAP_BOTH)
        m.check()
        assert np.array_equal(m.field(v.MAP_ENV)[0].cpu().numpy(), ref), t
    autotune.MapTuning(0, 0).apply(m)
    assert m.tile_z() == 8    # the default: X = 96 is a multiple of 8
    assert autotune.apply_cached_map(m, dims, path=path) == best
    assert autotune.tune_map(m, st, dims, path=path) == (best, {})
    m.close()
