"""The allocation-free EDT entry point (vedt_edt_noalloc).

Callers that must not allocate device memory while running -- a hard real-time control
loop, where cudaMalloc could stall the device past the cycle deadline, or a process whose
device memory belongs to another allocator -- use this entry point.  Its scratch is a
fixed array inside the library, so these tests check that its results equal the regular
vedt_compute_edt path on two calls in a row (the second call reuses the scratch the first
one left behind), and that grids too large for that array are refused.

This file is named so that pytest collects it last."""
import numpy as np
import pytest

from paper_2407_02363_b300 import synth


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
    assert v._lib.vedt_edt_noalloc(dummy, 0, 8, 8, dummy, dummy, None) == v.EINVAL
    assert v._lib.vedt_edt_noalloc(None, 8, 8, 8, dummy, dummy, None) == v.EINVAL


@pytest.mark.gpu
def test_noalloc_matches_regular_entry_point_twice():
    import torch
    v = _lib()
    cases = [((128, 128, 128), 0.01, 1), ((100, 77, 60), 0.003, 2)]
    for dims, density, seed in cases:
        occ = synth.random_occupancy(seed, dims, density)
        # the regular path (its own allocated scratch)
        m = v.Map(dims, 0.01)
        m.upload_occupancy(v.MAP_ENV, occ)
        m.compute_edt(v.MAP_ENV)
        ref_sq, ref_ix = m.field(v.MAP_ENV)
        m.close()
        # the allocation-free path, caller-owned input and outputs
        X, Y, Z = dims
        occ_d = torch.from_numpy(occ).cuda()
        sq = torch.full((Z, Y, X), -7, dtype=torch.int32, device="cuda")
        ix = torch.full((Z, Y, X), -7, dtype=torch.int32, device="cuda")
        s = torch.cuda.current_stream()
        v.edt_noalloc(occ_d, dims, sq, ix, stream=s)
        torch.cuda.synchronize()
        assert torch.equal(sq, ref_sq), "sqdist differs from vedt_compute_edt"
        assert torch.equal(ix, ref_ix), "nearest index differs from vedt_compute_edt"
