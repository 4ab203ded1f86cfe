"""Shared helpers for the GPU parity tests (imported only by tests)."""
import numpy as np

INT32_MAX = np.iinfo(np.int32).max


def lib():
    from paper_2407_02363_b300 import build
    build.build()
    from paper_2407_02363_b300 import vedt
    return vedt


def check_idx_valid(occ, sq, ix):
    """Every index names an occupied voxel at exactly the reported squared distance."""
    Z, Y, X = occ.shape
    flat = occ.reshape(-1)
    if not flat.any():
        assert (sq == INT32_MAX).all() and (ix == -1).all()
        return
    ixf = ix.reshape(-1).astype(np.int64)
    assert (ixf >= 0).all() and (ixf < occ.size).all()
    assert flat[ixf].all()
    lin = np.arange(occ.size, dtype=np.int64)
    vx, vy, vz = lin % X, (lin // X) % Y, lin // (X * Y)
    sx, sy, sz = ixf % X, (ixf // X) % Y, ixf // (X * Y)
    d = (vx - sx) ** 2 + (vy - sy) ** 2 + (vz - sz) ** 2
    assert np.array_equal(d, sq.reshape(-1).astype(np.int64))


def spheres_bitequal(a, b):
    """Bitwise equality of two sphere-result arrays (NaN payloads included)."""
    return a.dtype.itemsize == b.dtype.itemsize and np.array_equal(
        np.ascontiguousarray(a).view(np.uint8), np.ascontiguousarray(b).view(np.uint8))
