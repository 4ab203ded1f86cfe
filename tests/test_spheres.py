"""The OBB bounding-sphere generator (Sec. III-B) against closed forms: boxes of known
edges, rotation and translation invariance, the sphere count, diameter and spacing of the
rule, and the enclosure margin of the printed rule."""
import math

import numpy as np
import pytest

from paper_2407_02363_b300 import spheres, synth


def box_lattice(edges, step=0.005):
    """Lattice points filling an axis-aligned box centred at the origin, with extreme
    points exactly on its faces."""
    axes = [np.linspace(-e / 2, e / 2, int(round(e / step)) + 1) for e in edges]
    g = np.meshgrid(*axes, indexing="ij")
    return np.stack([a.ravel() for a in g], axis=1)


def rotation(seed):
    q = np.random.default_rng(seed).normal(size=4)
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_axis_aligned_box_and_its_sphere_row():
    edges = (0.2, 0.1, 0.5)                      # d1 = 0.1, d2 = 0.2, d3 = 0.5 once sorted
    box = spheres.obb_of_points(box_lattice(edges))
    np.testing.assert_allclose(box.half, [0.05, 0.1, 0.25], atol=1e-12)
    np.testing.assert_allclose(box.centre, 0.0, atol=1e-12)
    np.testing.assert_allclose(np.abs(box.axes), np.eye(3)[:, [1, 0, 2]], atol=1e-9)
    assert np.linalg.det(box.axes) > 0
    c, r = spheres.obb_spheres(box)
    D = math.sqrt(0.1 ** 2 + 0.2 ** 2)
    assert r == pytest.approx(D / 2, abs=1e-12)
    assert len(c) == math.ceil(0.5 / D + 1) == 4
    # on the long axis, from end face to end face, evenly spaced
    np.testing.assert_allclose(c[:, :2], 0.0, atol=1e-9)
    np.testing.assert_allclose(np.sort(c[:, 2]), np.linspace(-0.25, 0.25, 4), atol=1e-9)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_rotation_and_translation_invariance(seed):
    p = box_lattice((0.08, 0.3, 0.12))
    R, t = rotation(seed), np.array([0.3, -1.0, 2.0]) * seed
    a = spheres.obb_of_points(p)
    b = spheres.obb_of_points(p @ R.T + t)
    np.testing.assert_allclose(b.half, a.half, atol=1e-9)
    np.testing.assert_allclose(b.centre, R @ a.centre + t, atol=1e-9)
    np.testing.assert_allclose(np.abs(np.sum(b.axes * (R @ a.axes), axis=0)), 1.0, atol=1e-9)
    ca, ra = spheres.obb_spheres(a)
    cb, rb = spheres.obb_spheres(b)
    assert ra == pytest.approx(rb, abs=1e-12) and len(ca) == len(cb)
    # the rows match as sets (the long axis' sign is free)
    moved = ca @ R.T + t
    d = np.linalg.norm(moved[:, None, :] - cb[None, :, :], axis=2)
    assert d.min(axis=1).max() < 1e-9


def test_points_lie_in_their_box():
    rng = np.random.default_rng(5)
    p = rng.normal(size=(4000, 3)) * [0.02, 0.05, 0.2] @ rotation(9).T + [1, 2, 3]
    box = spheres.obb_of_points(p)
    proj = (p - box.centre) @ box.axes
    assert (np.abs(proj) <= box.half + 1e-12).all()
    # each extent is reached by some point on both sides
    np.testing.assert_allclose(proj.max(axis=0), box.half, atol=1e-12)
    np.testing.assert_allclose(proj.min(axis=0), -box.half, atol=1e-12)


def test_enclosure_margin_of_the_printed_rule():
    """Every box point is within r + gap of a centre, and the corner halfway between two
    centres is exactly r + gap away: the printed rule leaves that margin uncovered."""
    hx, hy, hz = 0.04, 0.05, 0.175
    box = spheres.obb_of_points(box_lattice((2 * hx, 2 * hy, 2 * hz)))
    c, r = spheres.obb_spheres(box)
    assert r == pytest.approx(math.hypot(hx, hy), abs=1e-12)
    gap = spheres.enclosure_gap(box)
    s = 2 * hz / (len(c) - 1)
    assert gap == pytest.approx(math.hypot(2 * r, s) / 2 - r, abs=1e-15) and gap > 0
    corners = np.array([[x, y, z] for x in (-hx, hx) for y in (-hy, hy) for z in np.linspace(-hz, hz, 71)])
    d = np.linalg.norm(corners[:, None, :] - c[None, :, :], axis=2).min(axis=1)
    assert d.max() <= r + gap + 1e-12
    mid = np.array([hx, hy, -hz + s / 2])
    assert np.linalg.norm(c - mid, axis=1).min() == pytest.approx(r + gap, abs=1e-9)
    # the box's axis is covered, and so is each sphere's own cross-section (its corners
    # lie on the sphere)
    axis = np.stack([np.zeros(50), np.zeros(50), np.linspace(-hz, hz, 50)], 1)
    assert (np.linalg.norm(axis[:, None] - c[None], axis=2).min(axis=1) <= r + 1e-12).all()
    own = c + [hx, hy, 0.0]
    np.testing.assert_allclose(np.linalg.norm(own - c, axis=1), r, atol=1e-9)


def test_degenerate_boxes():
    # long edge shorter than the face diagonal: two spheres (d3 / D = 0.937)
    box = spheres.obb_of_points(box_lattice((0.2, 0.25, 0.3), 0.01))
    c, r = spheres.obb_spheres(box)
    assert len(c) == 2 and r == pytest.approx(math.hypot(0.2, 0.25) / 2, abs=1e-12)
    # a flat rectangle: d1 = 0, D = d2 = 0.2, d3 / D = 1.5 -> three spheres
    c, r = spheres.obb_spheres(spheres.obb_of_points(box_lattice((0.0, 0.2, 0.3), 0.01)))
    assert len(c) == 3 and r == pytest.approx(0.1, abs=1e-12)
    # a single point: no cross-section
    with pytest.raises(ValueError):
        spheres.obb_spheres(spheres.obb_of_points(np.zeros((1, 3))))
    with pytest.raises(ValueError):
        spheres.obb_of_points(np.zeros((0, 3)))


def test_capsule_links_of_the_synthetic_chain():
    chain = synth.make_chain(3, (0, 0, 0))
    models = synth.link_models(chain, 0.02)
    sm = spheres.sphere_model_obb(models)
    assert sorted(set(sm.link.tolist())) == list(range(1, 8))
    for k in range(1, 8):
        box = spheres.obb_of_points(models[k])
        # the long axis is the link's z axis; the cross-section is the capsule's diameter
        assert abs(box.axes[2, 2]) == pytest.approx(1.0, abs=1e-6)
        assert box.half[2] * 2 <= chain.lengths[k - 1] + 2 * chain.radius + 1e-6
        assert box.half[2] * 2 >= chain.lengths[k - 1] + 2 * chain.radius - 0.02
        n = int((sm.link == k).sum())
        d1, d2, d3 = 2 * box.half
        assert n == math.ceil(d3 / math.hypot(d1, d2) + 1)
        # every voxel of the link lies within its row's spheres plus the enclosure margin
        c = sm.local[sm.link == k]
        r = float(sm.radius[sm.link == k][0])
        d = np.linalg.norm(models[k][:, None, :].astype(np.float64) - c[None], axis=2).min(axis=1)
        assert d.max() <= r + spheres.enclosure_gap(box) + 1e-9
    assert sm.acm.tolist() == np.isin(sm.link, (1, 2, 3)).tolist()
