"""GPU parity of the exact EDT (Sec. III-C, Alg. 1) against the CPU oracle, through the
C ABI: squared distances bit-exact everywhere, every nearest index valid (ties may pick
another equally near voxel)."""
import numpy as np
import pytest

import oracle
from paper_2407_02363_b300 import synth
from gpu_helpers import INT32_MAX, check_idx_valid, lib

pytestmark = pytest.mark.gpu


def run_gpu_edt(occ_env, occ_self=None, which=None, bands=0, tile_z=0):
    v = lib()
    Z, Y, X = occ_env.shape
    m = v.Map((X, Y, Z), 0.01)
    m.set_bands(bands)
    m.set_tile_z(tile_z)
    m.upload_occupancy(v.MAP_ENV, occ_env)
    if occ_self is not None:
        m.upload_occupancy(v.MAP_SELF, occ_self)
    w = which if which is not None else (v.MAP_BOTH if occ_self is not None else v.MAP_ENV)
    m.compute_edt(w)
    m.check()
    out = []
    for g in (v.MAP_ENV, v.MAP_SELF):
        if w & g:
            sq, ix = m.field(g)
            out.append((sq.cpu().numpy(), ix.cpu().numpy()))
    m.close()
    return out


def assert_parity(occ, sq, ix):
    osq, _ = oracle.edt(occ)
    assert np.array_equal(sq, osq), f"{int((sq != osq).sum())} voxels differ"
    check_idx_valid(occ, sq, ix)


CASES = [
    ((16, 16, 16), 0.001), ((16, 16, 16), 0.05), ((16, 16, 16), 0.5),
    ((64, 64, 64), 0.02), ((37, 50, 29), 0.01), ((100, 3, 70), 0.02),
    ((33, 65, 17), 0.3), ((200, 1, 1), 0.02), ((1, 300, 1), 0.02), ((1, 1, 256), 0.02),
    ((256, 7, 9), 0.005), ((31, 256, 40), 0.001), ((96, 64, 255), 0.0005),
    ((128, 128, 128), 0.0001),
]


@pytest.mark.parametrize("dims,density", CASES)
def test_edt_small_mode(dims, density):
    occ = synth.random_occupancy(hash(dims) % 1000, dims, density)
    occ2 = synth.random_occupancy(hash(dims) % 1000 + 1, dims, density * 0.5)
    (sq, ix), (sq2, ix2) = run_gpu_edt(occ, occ2)
    assert_parity(occ, sq, ix)
    assert_parity(occ2, sq2, ix2)


LARGE = [((300, 40, 20), 0.01), ((260, 260, 8), 0.002), ((40, 20, 700), 0.003),
         ((512, 64, 64), 0.001), ((70, 513, 33), 0.02), ((1024, 2, 3), 0.01)]


@pytest.mark.parametrize("dims,density", LARGE)
def test_edt_large_mode(dims, density):
    occ = synth.random_occupancy(7 + sum(dims), dims, density)
    (sq, ix), = run_gpu_edt(occ)
    assert_parity(occ, sq, ix)


@pytest.mark.parametrize("tile_z", [8, 32])
@pytest.mark.parametrize("bands", [1, 2, 4, 8])
def test_edt_band_count_does_not_change_the_field(bands, tile_z):
    """Bands per line (Alg. 1's m2 / m3, the ablation of Tab. 2) and the pass-Z tile shape
    change speed only: lines shorter than, equal to and longer than a band multiple,
    sparse and dense, X a multiple of 8 and not (8 x 4 patches cut by the grid's edge),
    Y no multiple of 4 (a ragged last patch)."""
    for dims, dens in (((96, 70, 37), 0.01), ((256, 33, 256), 0.002), ((45, 256, 129), 0.3), ((7, 5, 3), 0.2)):
        occ = synth.random_occupancy(31 + bands + sum(dims), dims, dens)
        (sq, ix), = run_gpu_edt(occ, bands=bands, tile_z=tile_z)
        assert_parity(occ, sq, ix)


def test_tile_z_default_and_values():
    """The default pass-Z tile is 8 x 4 when X is a multiple of 8, else 32 x 1, for grids
    up to 256 and above; 8 and 32 are settable, nothing else."""
    v = lib()
    maps = {dims: v.Map(dims, 0.01) for dims in ((64, 30, 20), (45, 30, 20), (304, 8, 8), (300, 8, 8))}
    assert [m.tile_z() for m in maps.values()] == [8, 32, 8, 32]
    for dims, m in maps.items():
        default = m.tile_z()
        for tz in (8, 32):
            m.set_tile_z(tz)
            assert m.tile_z() == tz
        m.set_tile_z(0)
        assert m.tile_z() == default
        for bad in (4, 16, -1, 64):
            with pytest.raises(v.VedtError):
                m.set_tile_z(bad)
        m.close()


@pytest.mark.parametrize("tile_z", [8, 32])
@pytest.mark.parametrize("bands", [4, 8])
def test_edt_band_count_large_mode(bands, tile_z):
    """Grids above 256 (16-bit row sites, 32-bit 2-D sites): lines longer than one TMA box
    (z = 300: two boxes, the second read past the grid), Y no multiple of 4, X no multiple
    of 8, at both pass-Z tile shapes."""
    for dims, dens in (((300, 40, 250), 0.002), ((40, 513, 20), 0.01), ((100, 30, 300), 0.01)):
        occ = synth.random_occupancy(41 + bands + sum(dims), dims, dens)
        (sq, ix), = run_gpu_edt(occ, bands=bands, tile_z=tile_z)
        assert_parity(occ, sq, ix)


def test_set_bands_rejects_values_outside_the_mode():
    v = lib()
    small, large = v.Map((64, 64, 64), 0.01), v.Map((300, 8, 8), 0.01)
    for m, bad in ((small, (3, 16, -1)), (large, (1, 2, 3, 16))):
        for b in bad:
            with pytest.raises(v.VedtError):
                m.set_bands(b)
    small.set_bands(1)
    large.set_bands(8)
    small.set_bands(0)
    small.close()
    large.close()


@pytest.mark.parametrize("dims", [(16, 16, 16), (300, 20, 10)])
def test_edt_empty_and_full(dims):
    Z = dims[2]
    empty = np.zeros((Z, dims[1], dims[0]), np.uint8)
    full = np.ones_like(empty)
    (sq, ix), (sq2, ix2) = run_gpu_edt(empty, full)
    assert (sq == INT32_MAX).all() and (ix == -1).all()
    assert (sq2 == 0).all() and np.array_equal(ix2.reshape(-1), np.arange(full.size))


def test_edt_single_site_and_empty_slices():
    dims = (64, 48, 40)
    for site in [(0, 0, 0), (63, 47, 39), (31, 0, 20)]:
        occ = synth.sites_occupancy(dims, [site])
        (sq, ix), = run_gpu_edt(occ)
        Z, Y, X = occ.shape
        gz, gy, gx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
        expect = (gx - site[0]) ** 2 + (gy - site[1]) ** 2 + (gz - site[2]) ** 2
        assert np.array_equal(sq, expect)
        assert (ix == site[0] + X * (site[1] + Y * site[2])).all()


def test_edt_max_int_range_corners():
    """Opposite corners of a 256^3 grid: the largest squared distances of small mode."""
    dims = (256, 256, 256)
    occ = synth.sites_occupancy(dims, [(0, 0, 0)])
    (sq, ix), = run_gpu_edt(occ)
    assert sq[255, 255, 255] == 3 * 255 * 255
    assert_parity(occ, sq, ix)


def test_edt_full_size_256_and_512():
    for dims, dens in (((256, 256, 256), 0.02), ((512, 512, 512), 0.003), ((512, 512, 128), 0.0005),
                       ((192, 192, 128), 0.002)):
        occ = synth.random_occupancy(5, dims, dens)
        (sq, ix), = run_gpu_edt(occ)
        assert_parity(occ, sq, ix)
        del occ, sq, ix


def test_edt_repeat_is_deterministic_and_independent_of_other_grid():
    dims = (96, 80, 72)
    occ = synth.random_occupancy(11, dims, 0.01)
    other = synth.random_occupancy(12, dims, 0.2)
    (a, ai), = run_gpu_edt(occ, which=None)
    (b, bi), (_, _) = run_gpu_edt(occ, other)
    assert np.array_equal(a, b) and np.array_equal(ai, bi)


def test_edt_random_sweep_of_shapes_densities_and_bands():
    """Seeded sweep: ragged dims (not multiples of 32), densities from one site to dense,
    every band count of the mode, small and large mode."""
    rng = np.random.default_rng(2024)
    for case in range(40):
        large = case % 5 == 4
        if large:
            dims = (int(rng.integers(257, 400)), int(rng.integers(1, 40)), int(rng.integers(1, 40)))
            dims = tuple(np.roll(dims, int(rng.integers(0, 3))))
            bands = int(rng.choice([0, 4, 8]))
        else:
            dims = tuple(int(d) for d in rng.integers(1, 97, 3))
            bands = int(rng.choice([0, 1, 2, 4, 8]))
        dens = float(10 ** rng.uniform(-4, -0.3))
        occ = synth.random_occupancy(5000 + case, dims, dens)
        if occ.sum() == 0 and case % 2:
            occ.flat[int(rng.integers(0, occ.size))] = 1
        (sq, ix), = run_gpu_edt(occ, bands=bands)
        if occ.any():
            assert_parity(occ, sq, ix)
        else:
            assert (sq == INT32_MAX).all() and (ix == -1).all()
