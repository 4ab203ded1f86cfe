"""Band junctions of EDT passes Y and Z, at every band count, against the oracle.

The envelope passes build one stack per band and join the bands at their junctions; the
inputs below are built so that the joins do the most work:
* every position owns itself: every line's envelope holds all of its positions, so each
  junction keeps both neighbours' whole stacks;
* a cascade: most positions hold far sites and one late position a near site that beats
  them over the whole line, so the repair pops every earlier band empty, one after the
  other;
* alternating near and far sites with empty stretches that put junctions next to empty
  bands;
and random single sites per line as a control.  Squared distances must equal the oracle
element by element and every index must be valid."""
import numpy as np
import pytest

from gpu_helpers import check_idx_valid, lib

pytestmark = pytest.mark.gpu


def _run(v, occ, bands, tile_z=0):
    import oracle
    Z, Y, X = occ.shape
    m = v.Map((X, Y, Z), 0.01)
    m.set_bands(bands)
    m.set_tile_z(tile_z)
    m.upload_occupancy(v.MAP_ENV, occ)
    m.compute_edt(v.MAP_ENV)
    m.check()
    sq, ix = (t.cpu().numpy() for t in m.field(v.MAP_ENV))
    m.close()
    osq, _ = oracle.edt(occ)
    bad = np.argwhere(sq != osq)
    assert bad.size == 0, (bands, len(bad), bad[:3])
    check_idx_valid(occ, sq, ix)


def _z_cases(X, Y, Z, rng):
    out = {}
    a = np.zeros((Z, Y, X), np.uint8)
    a[:, 0, 0] = 1                          # every slice: a site at the column origin
    out["own"] = a
    b = np.zeros((Z, Y, X), np.uint8)
    b[: Z * 3 // 4, Y - 1, X - 1] = 1       # far sites in the first three quarters
    b[Z - 10, 0, 0] = 1                     # one near site late in the line
    out["cascade"] = b
    c = np.zeros((Z, Y, X), np.uint8)
    for z in range(Z):
        if (z // 7) % 3 == 2:
            continue                        # empty stretches
        if z % 2:
            c[z, Y - 1, X - 1] = 1
        else:
            c[z, rng.integers(0, Y // 4), rng.integers(0, X // 4)] = 1
    out["alternate"] = c
    d = np.zeros((Z, Y, X), np.uint8)
    zs = rng.choice(Z, size=Z // 3, replace=False)
    d[zs, rng.integers(0, Y, zs.size), rng.integers(0, X, zs.size)] = 1
    out["random"] = d
    return out


@pytest.mark.parametrize("tile_z", [8, 32])
@pytest.mark.parametrize("bands", [1, 2, 4, 8])
def test_pass_z_junctions(bands, tile_z):
    """256-long z lines; x spans 256 so that the far sites of the cascade (in-plane
    distance 255) lose to the near site over the whole line.  Both pass-Z tile shapes."""
    v = lib()
    rng = np.random.default_rng(bands)
    for name, occ in _z_cases(256, 8, 256, rng).items():
        _run(v, occ, bands, tile_z)


@pytest.mark.parametrize("bands", [1, 2, 4, 8])
def test_pass_y_junctions(bands):
    """The same patterns along y (one slice per line family), long y lines."""
    v = lib()
    rng = np.random.default_rng(10 + bands)
    for name, occ in _z_cases(256, 8, 256, rng).items():
        _run(v, np.ascontiguousarray(occ.transpose(1, 0, 2)), bands)   # z <-> y


@pytest.mark.parametrize("bands", [1, 2, 4, 8])
def test_ragged_lines_junctions(bands):
    """Line lengths that leave short and empty last bands (n not a multiple of the band count)."""
    v = lib()
    rng = np.random.default_rng(20 + bands)
    for n in (7, 33, 129, 250):
        for occ in _z_cases(40, 24, n, rng).values():
            _run(v, occ, bands, 8)
            _run(v, occ, bands, 32)
            _run(v, np.ascontiguousarray(occ.transpose(1, 0, 2)), bands)
