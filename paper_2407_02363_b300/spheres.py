"""Bounding-sphere model of the robot from its link voxel models (Sec. III-B), computed
once offline:

  * an oriented bounding box (OBB) per link: centre, orientation and three half-edge
    lengths.  The paper does not say how the box is fitted; here its axes are the
    principal axes of the link's points (eigenvectors of their covariance) and its extent
    along each axis is the points' range;
  * for box edge lengths d1 <= d2 <= d3, spheres of diameter D = sqrt(d1^2 + d2^2) (the
    diagonal of the box's smallest face), ceil(d3 / D + 1) of them, centred on the box's
    long axis and spaced evenly from one end face to the other.

The paper states that this row of spheres encloses the box.  It does along the box's
axis and at every sphere's own cross-section, where the face diagonal is the diameter;
between two centres a distance s apart the cross-section's corners lie
sqrt(D^2 + s^2) / 2 from the nearer centre, outside by at most that minus D / 2.  The
model follows the printed rule and `enclosure_gap` reports that margin.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .synth import SphereModel


@dataclass(frozen=True)
class OBB:
    centre: np.ndarray   # (3,) in the frame of the points
    axes: np.ndarray     # (3, 3) columns: unit box axes, by ascending extent; right-handed
    half: np.ndarray     # (3,) half-edge lengths, ascending


def obb_of_points(points) -> OBB:
    """Principal-axis oriented bounding box of a point set (k >= 1 points, float64)."""
    p = np.asarray(points, np.float64).reshape(-1, 3)
    if p.shape[0] == 0:
        raise ValueError("empty point set")
    mu = p.mean(axis=0)
    q = p - mu
    _, V = np.linalg.eigh(q.T @ q)
    proj = q @ V
    lo, hi = proj.min(axis=0), proj.max(axis=0)
    half = (hi - lo) / 2.0
    centre = mu + V @ ((lo + hi) / 2.0)
    order = np.argsort(half, kind="stable")
    V = V[:, order]
    half = half[order]
    if np.linalg.det(V) < 0:
        V[:, 0] = -V[:, 0]
    return OBB(centre=centre, axes=V, half=half)


def obb_spheres(box: OBB):
    """(centres (n, 3), radius) of the sphere row of one box: diameter D = sqrt(d1^2 +
    d2^2), n = ceil(d3 / D + 1), centres evenly spaced on the long axis with the first and
    last at the centres of the end faces (one sphere at the box centre if d3 = 0)."""
    d1, d2, d3 = (2.0 * box.half).tolist()
    D = math.hypot(d1, d2)
    if D == 0.0:
        raise ValueError("box with a degenerate cross-section (all points on a line)")
    n = int(math.ceil(d3 / D + 1.0))
    t = np.linspace(-d3 / 2.0, d3 / 2.0, n) if n > 1 else np.zeros(1)
    centres = box.centre[None, :] + t[:, None] * box.axes[:, 2][None, :]
    return centres, D / 2.0


def enclosure_gap(box: OBB) -> float:
    """How far the box pokes out of its sphere row: the largest distance from a box point
    to the union of the spheres, reached at the cross-section corners halfway between two
    centres (0 for a single sphere on a box with d3 = 0)."""
    centres, r = obb_spheres(box)
    if len(centres) < 2:
        return 0.0
    s = 2.0 * box.half[2] / (len(centres) - 1)
    return math.hypot(2.0 * r, s) / 2.0 - r


def sphere_model_obb(link_models, acm_links=(1, 2, 3)) -> SphereModel:
    """Sphere model of links 1..n from their voxel models (index 0, the static body, is an
    obstacle, not a controlled link): each link's OBB in its own frame and its sphere row."""
    links, local, radius = [], [], []
    for k in range(1, len(link_models)):
        box = obb_of_points(link_models[k])
        c, r = obb_spheres(box)
        links.extend([k] * len(c))
        local.extend(c.tolist())
        radius.extend([r] * len(c))
    links = np.asarray(links, dtype=np.int32)
    return SphereModel(link=links, local=np.asarray(local, dtype=np.float64),
                       radius=np.asarray(radius, dtype=np.float32), acm=np.isin(links, np.asarray(acm_links)))
