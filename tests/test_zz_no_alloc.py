"""The allocation-free EDT entry point (vedt_edt_noalloc).

Callers that must not allocate device memory while running -- a hard real-time control
loop, where cudaMalloc could stall the device past the cycle deadline, or a process whose
device memory belongs to another allocator -- use this entry point.  Its scratch is a
fixed array inside the library, so these tests check its results against the oracle
(squared distances element by element, every nearest index valid) and against the
regular vedt_compute_edt path, on calls in a row (each call reuses the scratch the
previous one left behind), at the size limit of that array, and on the index-checked
build; and that grids too large for the array and malformed buffers are refused.

This file is named so that pytest collects it last."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2407_02363_b300 import synth
from gpu_helpers import check_idx_valid

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _lib():
    from paper_2407_02363_b300 import build
    build.build()
    from paper_2407_02363_b300 import vedt
    return vedt


def test_noalloc_refuses_grids_beyond_its_scratch():
    v = _lib()
    import ctypes
    dummy = ctypes.c_void_p(16)   # never dereferenced: the size check comes first
    assert v._lib.vedt_edt_noalloc(dummy, 257, 8, 8, dummy, dummy, None) == v.ENOTSUP
    assert v._lib.vedt_edt_noalloc(dummy, 160, 128, 128, dummy, dummy, None) == v.ENOTSUP   # 160 pads to 160; 2.6M > 2^21
    assert v._lib.vedt_edt_noalloc(dummy, 33, 256, 256, dummy, dummy, None) == v.ENOTSUP    # pads to 64: 2^22
    assert v._lib.vedt_edt_noalloc(dummy, 0, 8, 8, dummy, dummy, None) == v.EINVAL
    assert v._lib.vedt_edt_noalloc(None, 8, 8, 8, dummy, dummy, None) == v.EINVAL


def test_noalloc_binding_checks_buffers():
    """The binding refuses wrong dtypes, sizes and non-CUDA tensors before any call, so a
    malformed buffer can never let the kernels write past it."""
    import torch
    v = _lib()
    dims = (8, 8, 8)
    good_occ = torch.zeros(512, dtype=torch.uint8)
    good_out = torch.zeros(512, dtype=torch.int32)
    with pytest.raises(ValueError):   # int64 field
        v.edt_noalloc(good_occ, dims, torch.zeros(512, dtype=torch.int64), good_out)
    with pytest.raises(ValueError):   # too small
        v.edt_noalloc(good_occ, dims, torch.zeros(511, dtype=torch.int32), good_out)
    with pytest.raises(ValueError):   # occupancy of the wrong size
        v.edt_noalloc(torch.zeros(500, dtype=torch.uint8), dims, good_out, good_out)
    with pytest.raises(ValueError):   # not contiguous
        v.edt_noalloc(good_occ, dims, torch.zeros(1024, dtype=torch.int32)[::2], good_out)
    with pytest.raises(ValueError):   # host tensors
        v.edt_noalloc(good_occ, dims, good_out, good_out)


def _regular(v, occ, dims):
    m = v.Map(dims, 0.01)
    m.upload_occupancy(v.MAP_ENV, occ)
    m.compute_edt(v.MAP_ENV)
    sq, ix = m.field(v.MAP_ENV)
    sq, ix = sq.clone(), ix.clone()
    m.check()
    m.close()
    return sq, ix


def _run_cases(cases):
    import torch
    import oracle
    v = _lib()
    for dims, density, seed in cases:
        occ = synth.random_occupancy(seed, dims, density)
        ref_sq, ref_ix = _regular(v, occ, dims)
        X, Y, Z = dims
        occ_d = torch.from_numpy(occ).cuda()
        sq = torch.full((Z, Y, X), -7, dtype=torch.int32, device="cuda")
        ix = torch.full((Z, Y, X), -7, dtype=torch.int32, device="cuda")
        v.edt_noalloc(occ_d, dims, sq, ix, stream=torch.cuda.current_stream())
        osq, _ = oracle.edt(occ)
        got_sq, got_ix = sq.cpu().numpy(), ix.cpu().numpy()
        assert np.array_equal(got_sq, osq), f"{dims}: sqdist differs from the oracle"
        check_idx_valid(occ, got_sq, got_ix)
        assert torch.equal(sq, ref_sq), f"{dims}: sqdist differs from vedt_compute_edt"
        assert torch.equal(ix, ref_ix), f"{dims}: nearest index differs from vedt_compute_edt"


@pytest.mark.gpu
def test_noalloc_matches_regular_entry_point_twice():
    """Two calls in a row of different shapes, then the same shape again."""
    _run_cases([((128, 128, 128), 0.01, 1), ((100, 77, 60), 0.003, 2), ((128, 128, 128), 0.02, 3)])


@pytest.mark.gpu
def test_noalloc_at_the_scratch_limit():
    """Grids that fill the 2^21 padded voxels exactly, with 256-long lines (the longest TMA
    box) along y and z, and one with odd Y * Z and a ragged x."""
    _run_cases([((32, 256, 256), 0.004, 4), ((256, 128, 64), 0.004, 5), ((250, 127, 63), 0.01, 6)])


@pytest.mark.gpu
def test_noalloc_on_the_index_checked_build():
    """The same calls on libvedt_debug.so, whose passes check every index they compute; a
    flagged index would make vedt_edt_noalloc return VEDT_ECUDA (the call reads its error
    word back)."""
    from paper_2407_02363_b300 import build
    build.build(debug=True)
    env = dict(os.environ, VEDT_DEBUG_BOUNDS="1")
    code = ("import sys; sys.path.insert(0, 'tests'); import test_zz_no_alloc as t; "
            "from paper_2407_02363_b300 import vedt; assert 'index checks' in vedt.version(); "
            "t._run_cases([((128, 128, 128), 0.01, 1), ((100, 77, 60), 0.003, 2), ((32, 256, 256), 0.004, 4)]); "
            "print('ok')")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
