"""CPU-side checks of the C ABI: the library loads, exports every entry point that
include/*.h declares, validates arguments on the host before touching the GPU, and its
host forward kinematics agrees with the oracle's."""
import glob
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2407_02363_b300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def v():
    from paper_2407_02363_b300 import build
    build.build()
    from paper_2407_02363_b300 import vedt
    return vedt


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(vedt_[a-z0-9_]+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(v):
    declared = _declared()
    assert "vedt_compute_edt" in declared and "vedt_query_spheres" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", v.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (vedt_[a-z0-9_]+)", out))
    assert declared <= exported, sorted(declared - exported)


def test_status_strings(v):
    assert v.status_string(0) == "ok"
    assert "invalid" in v.status_string(-1)
    assert v.version().startswith("vedt")


@pytest.mark.parametrize("dims,vs", [((0, 4, 4), 0.01), ((4, 4, 1025), 0.01), ((4, 4, 4), 0.0),
                                     ((4, 4, 4), -1.0), ((4, 4, 4), float("nan"))])
def test_map_create_rejects_bad_arguments(v, dims, vs):
    with pytest.raises(v.VedtError) as e:
        v.Map(dims, vs)
    assert e.value.status == v.EINVAL


def test_null_handle_calls_rejected(v):
    import ctypes
    L = v._lib
    assert L.vedt_clear(None, 3) == v.EINVAL
    assert L.vedt_compute_edt(None, 3) == v.EINVAL
    assert L.vedt_insert_pointcloud(None, None, 10, None, 0, None) == v.EINVAL
    assert L.vedt_query_spheres(None, None, None, 1, 3, None) == v.EINVAL
    assert L.vedt_map_destroy(None) == v.OK
    assert L.vedt_check(None) == v.EINVAL
    assert L.vedt_fk(None, None, None) == v.EINVAL
    assert L.vedt_map_set_bands(None, 4) == v.EINVAL
    assert L.vedt_map_set_incremental(None, 1) == v.EINVAL
    assert L.vedt_map_edt_recomputed(None, 3, None) == v.EINVAL
    assert L.vedt_insert_pointcloud_masked(None, None, 10, None, 0, None, None) == v.EINVAL
    assert L.vedt_sor_filter(None, None, 10, 8, 1.0, None) == v.EINVAL
    assert L.vedt_sor_stats(None, None, None) == v.EINVAL
    assert L.vedt_sor_mean_distances(None, None) == v.EINVAL
    assert L.vedt_sor_destroy(None) == v.OK
    assert L.vedt_map_set_logodds(None, 1, 9, 4, -20, 40, 15) == v.EINVAL
    assert L.vedt_update_occupancy(None) == v.EINVAL
    assert L.vedt_mlp_get_state(None, None, None, None, 10, None) == v.EINVAL
    assert L.vedt_mlp_set_state(None, None, None, None, 10, 0) == v.EINVAL
    out = ctypes.c_void_p()
    for bad in (0, -5):
        assert L.vedt_sor_create(bad, None, ctypes.byref(out)) == v.EINVAL


def test_fk_matches_oracle(v, oracle_mod):
    chain = synth.make_chain(3, (1.28, 1.28, 1.28))
    for q in synth.joint_states(4, 20):
        P = v.fk(chain, q)
        R = oracle_mod.fk(chain, q)
        assert np.abs(P - R).max() < 1e-12
        # same operation order on both sides: identical fp32 poses
        assert np.array_equal(P.astype(np.float32), R.astype(np.float32))


def test_sphere_centres_bitequal_to_oracle(v, oracle_mod):
    """vedt_sphere_centres (Alg. 2 line 8 behind the ABI) rounds the same fp64 sums as the
    oracle's sphere_centres, in the same order: identical fp32 centres, one by one and
    batched."""
    chain = synth.make_chain(3, (1.28, 1.28, 1.28))
    spheres = synth.sphere_model(chain)
    rng = np.random.default_rng(5)
    off_axis = synth.SphereModel(link=np.array([0, 1, 4, 7, 7], np.int32), local=rng.uniform(-0.2, 0.2, (5, 3)),
                                 radius=np.full(5, 0.05, np.float32))
    qs = synth.joint_states(6, 12)
    for sph in (spheres, off_axis):
        batch = v.sphere_centres_batch(chain, sph, qs)
        per_cycle = v.SphereCentres(chain, sph)   # the cached per-cycle form
        for i, q in enumerate(qs):
            want = oracle_mod.sphere_centres(chain, sph, q)
            got = v.sphere_centres(chain, sph, q)
            assert got.dtype == np.float32 and np.array_equal(got, want)
            assert np.array_equal(batch[i], want)
            cyc = per_cycle(q)
            assert cyc is per_cycle.out and np.array_equal(cyc, want)   # one buffer, overwritten


def test_sphere_centres_rejects_bad_arguments(v):
    import ctypes
    chain = synth.make_chain(3, (1.28, 1.28, 1.28))
    c = v.make_chain(chain)
    q = np.zeros(7)
    loc = np.zeros((2, 3))
    out = np.zeros((2, 3), np.float32)
    L = v._lib
    for links in (np.array([0, 8], np.int32), np.array([-1, 1], np.int32)):
        assert L.vedt_sphere_centres(ctypes.byref(c), v._np_ptr(q), 2, v._np_ptr(links), v._np_ptr(loc),
                                     v._np_ptr(out)) == v.EINVAL
    ok = np.array([0, 7], np.int32)
    assert L.vedt_sphere_centres(None, v._np_ptr(q), 2, v._np_ptr(ok), v._np_ptr(loc), v._np_ptr(out)) == v.EINVAL
    assert L.vedt_sphere_centres(ctypes.byref(c), None, 2, v._np_ptr(ok), v._np_ptr(loc), v._np_ptr(out)) == v.EINVAL
    assert L.vedt_sphere_centres(ctypes.byref(c), v._np_ptr(q), -1, v._np_ptr(ok), v._np_ptr(loc),
                                 v._np_ptr(out)) == v.EINVAL
    assert L.vedt_sphere_centres(ctypes.byref(c), None, 0, None, None, None) == v.OK
    assert L.vedt_sphere_centres_batch(ctypes.byref(c), v._np_ptr(q), -1, 2, v._np_ptr(ok), v._np_ptr(loc),
                                       v._np_ptr(out)) == v.EINVAL


def test_binding_refuses_to_load_without_the_library(tmp_path):
    """No CPU fallback: a copy of the package without libvedt.so fails at import."""
    import shutil
    pkg = tmp_path / "paper_2407_02363_b300"
    pkg.mkdir()
    src = os.path.join(ROOT, "paper_2407_02363_b300")
    for f in ("__init__.py", "vedt.py"):
        shutil.copy(os.path.join(src, f), pkg / f)
    code = "import paper_2407_02363_b300.vedt"
    r = subprocess.run([os.sys.executable, "-c", code], cwd=tmp_path, capture_output=True, text=True)
    assert r.returncode != 0
    assert "libvedt.so not built" in r.stderr

def test_build_tracks_every_source_and_header():
    """A change to any kernel source or header rebuilds the library: the up-to-date check
    covers the .cu sources, the .h and .cuh headers beside them and the public header."""
    import glob
    import os
    from paper_2407_02363_b300 import build
    deps = set(build._deps())
    csrc = os.path.join(os.path.dirname(build.__file__), "csrc")
    for pattern in ("*.cu", "*.cuh", "*.h"):
        files = glob.glob(os.path.join(csrc, pattern))
        assert files and set(files) <= deps, pattern
    assert any(p.endswith(os.path.join("include", "vedt.h")) for p in deps)
