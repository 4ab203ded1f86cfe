"""Autotuner: cache keys, winner selection and cache round trip on the CPU; on the GPU,
a real sweep over a batch whose results must not depend on the chosen launch shape."""
import numpy as np
import pytest

from paper_2407_02363_b300 import autotune, synth


def test_signature_is_order_independent():
    a = autotune.signature("B300", [(64, 80, 90), (100, 100, 100)])
    b = autotune.signature("B300", [(100, 100, 100), (64, 80, 90)])
    c = autotune.signature("B300", [(100, 100, 100), (64, 80, 91)])
    d = autotune.signature("H100", [(100, 100, 100), (64, 80, 90)])
    assert a == b and a != c and a != d


def test_pick_smallest_and_cache_roundtrip(tmp_path):
    t1, t2, t3 = autotune.Tuning(1, 0, 32), autotune.Tuning(1, 4, 8), autotune.Tuning(0, 0, 32)
    assert autotune.pick({t1: 2.0, t2: 1.5, t3: 3.0}) == t2
    p = str(tmp_path / "c.json")
    autotune.store_cache({"k": {"tuning": {"persistent": 1, "ctas_per_sm": 4, "rows_per_item": 8}}}, p)
    assert autotune.load_cache(p)["k"]["tuning"]["ctas_per_sm"] == 4
    assert autotune.load_cache(str(tmp_path / "missing.json")) == {}


@pytest.mark.gpu
def test_tune_sweeps_and_results_do_not_change(tmp_path):
    import torch

    import oracle
    from gpu_helpers import lib
    v = lib()
    dims_list = synth.batch_dims(5, n_maps=6)
    maps = [v.Map(tuple(int(x) for x in d), 0.02) for d in dims_list]
    occs = []
    for i, (m, d) in enumerate(zip(maps, dims_list)):
        o = synth.random_occupancy(i, tuple(d), 0.002)
        m.upload_occupancy(v.MAP_ENV, o)
        m.upload_occupancy(v.MAP_SELF, o)
        occs.append(o)
    s = torch.cuda.Stream()
    b = v.Batch(maps, stream=s)
    cands = [(0, 0, 32), (1, 0, 32), (1, 2, 8)]
    path = str(tmp_path / "tune.json")
    best, times = autotune.tune(b, s, dims_list, candidates=cands, reps=2, path=path)
    assert len(times) == 3 and best in times and all(t > 0 for t in times.values())
    again, t2 = autotune.tune(b, s, dims_list, candidates=cands, path=path)
    assert again == best and t2 == {}           # served from the cache
    b.compute_edt()
    b.check()
    for m, o in zip(maps, occs):
        sq = m.field(v.MAP_SELF)[0].cpu().numpy()
        assert np.array_equal(sq, oracle.edt(o)[0])
    b.close()
