"""Seeded synthetic inputs for the distance-map pipeline.

This module only *draws* inputs: point clouds, occupancy grids, kinematic chains,
offline link voxel models, sphere models and joint states. It contains none of the
method's arithmetic (no voxel insertion, no distance transform, no forward
kinematics, no sphere query), so the CUDA path and the CPU oracle can both consume
exactly the same inputs without sharing any computation.

The workloads stand in for the paper's live sensor data (Sec. IV-A: Tiago arm,
ASUS Xtion depth camera at 30 Hz), which is not available here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "GridSpec", "Chain", "SphereModel",
    "random_occupancy", "sites_occupancy", "surface_cloud", "CameraScene",
    "make_chain", "capsule_points", "box_shell_points", "link_models",
    "sphere_model", "joint_states", "joint_trajectory", "batch_dims",
]


@dataclass(frozen=True)
class GridSpec:
    """A voxel grid: dims = (X, Y, Z) voxels, cubic voxels of edge `voxel_size` metres,
    world position of the grid's min corner = `origin`."""
    dims: tuple
    voxel_size: float
    origin: tuple = (0.0, 0.0, 0.0)

    @property
    def extent(self):
        return tuple(d * self.voxel_size for d in self.dims)

    @property
    def n_voxels(self):
        return int(self.dims[0]) * int(self.dims[1]) * int(self.dims[2])


# ----------------------------------------------------------------------------------
# Occupancy grids for EDT-only tests (layout [Z][Y][X], x fastest)
# ----------------------------------------------------------------------------------

def random_occupancy(seed: int, dims, density: float) -> np.ndarray:
    """Bernoulli(density) uint8 occupancy grid of shape (Z, Y, X)."""
    X, Y, Z = dims
    rng = np.random.default_rng(seed)
    return (rng.random((Z, Y, X)) < density).astype(np.uint8)


def sites_occupancy(dims, sites) -> np.ndarray:
    """Grid with exactly the given (x, y, z) voxels occupied."""
    X, Y, Z = dims
    g = np.zeros((Z, Y, X), dtype=np.uint8)
    for (x, y, z) in sites:
        g[z, y, x] = 1
    return g


# ----------------------------------------------------------------------------------
# Point clouds
# ----------------------------------------------------------------------------------

def _box_surface(rng, centre, half, n):
    """n points uniform by area on the surface of an axis-aligned box."""
    hx, hy, hz = half
    areas = np.array([hy * hz, hy * hz, hx * hz, hx * hz, hx * hy, hx * hy])
    face = rng.choice(6, size=n, p=areas / areas.sum())
    u = rng.uniform(-1.0, 1.0, size=(n, 2))
    p = np.empty((n, 3))
    ax = face // 2
    sgn = np.where(face % 2 == 0, -1.0, 1.0)
    for a in range(3):
        m = ax == a
        o = [b for b in range(3) if b != a]
        p[m, a] = sgn[m] * half[a]
        p[m, o[0]] = u[m, 0] * half[o[0]]
        p[m, o[1]] = u[m, 1] * half[o[1]]
    return p + np.asarray(centre)


def _sphere_surface(rng, centre, r, n):
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return np.asarray(centre) + r * v


def surface_cloud(seed: int, grid: GridSpec, n_points: int = 20_000, n_boxes: int = 3,
                  n_spheres: int = 3, noise: float = 0.003) -> np.ndarray:
    """Points sampled by surface area on random boxes (sides U[0.1, 0.4] m) and spheres
    (radius U[0.05, 0.2] m) whose centres are uniform in the grid's extent, plus
    isotropic N(0, noise) jitter.  Returns float32 (n_points, 3) world coordinates."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(grid.origin, dtype=np.float64)
    ext = np.asarray(grid.extent, dtype=np.float64)
    prims = []
    for _ in range(n_boxes):
        c = lo + rng.uniform(0, 1, 3) * ext
        half = rng.uniform(0.1, 0.4, 3) / 2
        area = 8 * (half[0] * half[1] + half[1] * half[2] + half[0] * half[2])
        prims.append(("box", c, half, area))
    for _ in range(n_spheres):
        c = lo + rng.uniform(0, 1, 3) * ext
        r = rng.uniform(0.05, 0.2)
        prims.append(("sphere", c, r, 4 * math.pi * r * r))
    areas = np.array([p[3] for p in prims])
    counts = rng.multinomial(n_points, areas / areas.sum())
    parts = []
    for p, k in zip(prims, counts):
        if p[0] == "box":
            parts.append(_box_surface(rng, p[1], p[2], k))
        else:
            parts.append(_sphere_surface(rng, p[1], p[2], k))
    pts = np.concatenate(parts, axis=0)
    pts = pts + rng.normal(scale=noise, size=pts.shape)
    rng.shuffle(pts, axis=0)
    return pts.astype(np.float32)


class CameraScene:
    """A static scene of boxes, spheres and vertical cylinders on a floor, seen by a
    pinhole depth camera (640x480, fx = fy = 525, cx = 319.5, cy = 239.5) placed outside
    the grid, plus a sphere obstacle of radius 0.3 m moving at 1 m/s (bouncing along x
    inside the grid).  `frame(i)` returns the first-hit point per pixel, subsampled to
    `n_points`, with N(0, noise) jitter, as float32 world coordinates."""

    W, H, F, CX, CY = 640, 480, 525.0, 319.5, 239.5

    def __init__(self, seed: int, grid: GridSpec, n_boxes=6, n_spheres=4, n_cyl=4,
                 n_points=300_000, noise=0.002, fps=30.0, speed=1.0, radius=0.3, resolution_scale=1.0):
        rng = np.random.default_rng(seed)
        if resolution_scale != 1.0:     # a denser sensor: more pixels, same field of view
            self.W = int(round(640 * resolution_scale))
            self.H = int(round(480 * resolution_scale))
            self.F = 525.0 * resolution_scale
            self.CX, self.CY = (self.W - 1) / 2, (self.H - 1) / 2
        self.seed, self.grid, self.n_points, self.noise = seed, grid, n_points, noise
        self.fps, self.speed, self.radius = fps, speed, radius
        lo = np.asarray(grid.origin, np.float64)
        ext = np.asarray(grid.extent, np.float64)
        self.lo, self.ext = lo, ext
        # camera outside the -y face, above the grid centre, looking at the centre
        eye = lo + ext * np.array([0.5, -0.35, 0.9])
        target = lo + ext * np.array([0.5, 0.55, 0.3])
        fwd = target - eye
        fwd /= np.linalg.norm(fwd)
        right = np.cross(fwd, np.array([0.0, 0.0, 1.0]))
        right /= np.linalg.norm(right)
        down = np.cross(fwd, right)
        u, v = np.meshgrid(np.arange(self.W, dtype=np.float64), np.arange(self.H, dtype=np.float64))
        d = (fwd[None, None, :] + ((u - self.CX) / self.F)[..., None] * right
             + ((v - self.CY) / self.F)[..., None] * down)
        d /= np.linalg.norm(d, axis=-1, keepdims=True)
        self.eye = eye
        self.dirs = d.reshape(-1, 3)
        # static primitives: a room (floor, back and side walls just inside the grid)
        t = np.full(self.dirs.shape[0], np.inf)
        floor_z = lo[2] + 0.05
        for axis, val in ((2, floor_z), (1, lo[1] + ext[1] - 0.05), (0, lo[0] + 0.05),
                          (0, lo[0] + ext[0] - 0.05)):
            with np.errstate(divide="ignore", invalid="ignore"):
                tp = (val - eye[axis]) / self.dirs[:, axis]
            hit = eye[None, :] + np.where(np.isfinite(tp), tp, 0)[:, None] * self.dirs
            inside = np.all((hit >= lo) & (hit <= lo + ext), axis=1)
            t = np.where((tp > 0) & np.isfinite(tp) & inside, np.minimum(t, tp), t)
        for _ in range(n_boxes):
            c = lo + ext * rng.uniform(0.15, 0.85, 3)
            c[2] = floor_z + rng.uniform(0.05, 0.4)
            half = rng.uniform(0.05, 0.25, 3)
            t = np.minimum(t, self._hit_box(c - half, c + half))
        for _ in range(n_spheres):
            c = lo + ext * rng.uniform(0.15, 0.85, 3)
            r = rng.uniform(0.05, 0.25)
            t = np.minimum(t, self._hit_sphere(c, r))
        for _ in range(n_cyl):
            c = lo + ext * rng.uniform(0.15, 0.85, 3)
            r = rng.uniform(0.03, 0.15)
            h = rng.uniform(0.3, 1.2)
            t = np.minimum(t, self._hit_cylinder(c[0], c[1], r, floor_z, floor_z + h))
        self.t_static = t
        self.obst_y = lo[1] + 0.6 * ext[1]
        self.obst_z = lo[2] + 0.45 * ext[2]

    def _hit_box(self, bmin, bmax):
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / self.dirs
            t1 = (bmin - self.eye) * inv
            t2 = (bmax - self.eye) * inv
        tn = np.nanmax(np.minimum(t1, t2), axis=1)
        tx = np.nanmin(np.maximum(t1, t2), axis=1)
        return np.where((tx >= tn) & (tx > 0), np.where(tn > 0, tn, np.inf), np.inf)

    def _hit_sphere(self, c, r):
        oc = self.eye - c
        b = self.dirs @ oc
        cc = oc @ oc - r * r
        disc = b * b - cc
        s = np.sqrt(np.maximum(disc, 0))
        t = -b - s
        return np.where((disc >= 0) & (t > 0), t, np.inf)

    def _hit_cylinder(self, cx, cy, r, z0, z1):
        ox, oy = self.eye[0] - cx, self.eye[1] - cy
        dx, dy = self.dirs[:, 0], self.dirs[:, 1]
        a = dx * dx + dy * dy
        b = ox * dx + oy * dy
        c = ox * ox + oy * oy - r * r
        disc = b * b - a * c
        with np.errstate(divide="ignore", invalid="ignore"):
            t = (-b - np.sqrt(np.maximum(disc, 0))) / a
        z = self.eye[2] + t * self.dirs[:, 2]
        ok = (disc >= 0) & (t > 0) & (z >= z0) & (z <= z1) & (a > 0)
        return np.where(ok, t, np.inf)

    def obstacle_centre(self, i: int):
        """Centre of the moving sphere at frame i (bouncing along x inside the grid)."""
        span = self.ext[0] - 2 * self.radius - 0.2
        s = (self.speed * i / self.fps) % (2 * span)
        x = self.lo[0] + self.radius + 0.1 + (s if s < span else 2 * span - s)
        return np.array([x, self.obst_y, self.obst_z])

    def frame(self, i: int) -> np.ndarray:
        rng = np.random.default_rng((self.seed, i))
        t = np.minimum(self.t_static, self._hit_sphere(self.obstacle_centre(i), self.radius))
        hit = np.flatnonzero(np.isfinite(t))
        if hit.size > self.n_points:
            hit = rng.choice(hit, size=self.n_points, replace=False)
        pts = self.eye + t[hit, None] * self.dirs[hit]
        pts = pts + rng.normal(scale=self.noise, size=pts.shape)
        return pts.astype(np.float32)


# ----------------------------------------------------------------------------------
# Robot: kinematic chain description, offline link voxel models, sphere model
# ----------------------------------------------------------------------------------

@dataclass
class Chain:
    """Serial chain.  Link 0 is the static body, placed in the world by `base` (3x4,
    rotation | translation).  Joint k (1..n) sits at `offsets[k-1]` (3x4) in the frame of
    link k-1 and rotates link k about the joint frame's z axis.  Link k (k >= 1) is a
    capsule of radius `radius` from its frame origin along +z for `lengths[k-1]` metres."""
    base: np.ndarray            # (3, 4) float64
    offsets: np.ndarray         # (n, 3, 4) float64
    lengths: np.ndarray         # (n,) float64
    radius: float = 0.04

    @property
    def n_joints(self):
        return int(self.offsets.shape[0])


def _rx(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]], dtype=np.float64)


def make_chain(seed: int, base_xyz, n_joints: int = 7, len_range=(0.1, 0.3),
               radius: float = 0.04, body_height: float = 0.05) -> Chain:
    """Random 7-DoF chain: link lengths U[len_range]; consecutive joint axes
    alternate between the parent's z axis and a perpendicular one."""
    rng = np.random.default_rng(seed)
    lengths = rng.uniform(len_range[0], len_range[1], n_joints)
    base = np.zeros((3, 4))
    base[:, :3] = np.eye(3)
    base[:, 3] = np.asarray(base_xyz, dtype=np.float64)
    offs = np.zeros((n_joints, 3, 4))
    for k in range(n_joints):
        if k == 0:
            offs[k, :, :3] = np.eye(3)
            offs[k, :, 3] = (0.0, 0.0, body_height)
        else:
            offs[k, :, :3] = _rx(math.pi / 2 if k % 2 == 1 else -math.pi / 2)
            offs[k, :, 3] = (0.0, 0.0, lengths[k - 1])
    return Chain(base=base, offsets=offs, lengths=lengths, radius=radius)


def capsule_points(length: float, radius: float, spacing: float) -> np.ndarray:
    """Offline binary model of a capsule link: lattice points (spacing `spacing`, lattice
    offset spacing/2) within `radius` of the segment (0,0,0)-(0,0,length).  float32 (k, 3)
    in the link frame."""
    r = radius
    ax = np.arange(-r + spacing / 2, r, spacing)
    az = np.arange(-r + spacing / 2, length + r, spacing)
    gx, gy, gz = np.meshgrid(ax, ax, az, indexing="ij")
    p = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)
    zc = np.clip(p[:, 2], 0.0, length)
    d2 = p[:, 0] ** 2 + p[:, 1] ** 2 + (p[:, 2] - zc) ** 2
    return p[d2 <= r * r].astype(np.float32)


def box_shell_points(lo, hi, spacing: float) -> np.ndarray:
    """Lattice points on the surface shell (one lattice layer) of an axis-aligned box."""
    axes = [np.arange(l + spacing / 2, h, spacing) for l, h in zip(lo, hi)]
    gx, gy, gz = np.meshgrid(*axes, indexing="ij")
    p = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)
    edge = np.zeros(p.shape[0], dtype=bool)
    for a in range(3):
        edge |= (p[:, a] <= axes[a][0] + 1e-9) | (p[:, a] >= axes[a][-1] - 1e-9)
    return p[edge].astype(np.float32)


def link_models(chain: Chain, voxel_size: float):
    """Offline link voxel models, sampled at voxel_size/2: index 0 is the static body
    (a torso box shell below the base plus a base plate), 1..n the capsule links."""
    s = voxel_size / 2
    torso = box_shell_points((-0.12, -0.12, -0.45), (0.12, 0.12, 0.0), s)
    plate = box_shell_points((-0.22, -0.22, -0.55), (0.22, 0.22, -0.45), s)
    models = [np.concatenate([torso, plate], axis=0)]
    for L in chain.lengths:
        models.append(capsule_points(float(L), chain.radius, s))
    return models


@dataclass
class SphereModel:
    """Bounding spheres: sphere i sits on link `link[i]` (1..n) at `local[i]` (link frame)
    with radius `radius[i]`.  `acm[i]` marks spheres whose link is adjacent to the
    self-obstacle links (allowed collisions): they are queried but masked in
    self-distance statistics."""
    link: np.ndarray
    local: np.ndarray
    radius: np.ndarray
    acm: np.ndarray = field(default=None)


def sphere_model(chain: Chain, n_spheres: int = 24, radius: float = 0.05,
                 acm_links=(1, 2, 3)) -> SphereModel:
    """24 spheres allotted to links in proportion to link length (at least one per link,
    largest remainder), evenly spaced along each link axis."""
    L = chain.lengths
    n = len(L)
    extra = n_spheres - n
    quota = extra * L / L.sum()
    cnt = np.floor(quota).astype(int)
    rem = extra - cnt.sum()
    order = np.argsort(-(quota - cnt), kind="stable")
    cnt[order[:rem]] += 1
    cnt += 1
    links, local = [], []
    for k in range(n):
        for i in range(cnt[k]):
            links.append(k + 1)
            local.append((0.0, 0.0, (i + 0.5) / cnt[k] * L[k]))
    links = np.array(links, dtype=np.int32)
    return SphereModel(link=links, local=np.array(local, dtype=np.float64),
                       radius=np.full(len(links), radius, dtype=np.float32),
                       acm=np.isin(links, np.asarray(acm_links)))


def joint_states(seed: int, n: int, n_joints: int = 7) -> np.ndarray:
    """(n, n_joints) float64 joint angles, uniform in [-pi, pi]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-math.pi, math.pi, size=(n, n_joints))


def joint_trajectory(seed: int, n_frames: int, n_joints: int = 7, fps: float = 30.0) -> np.ndarray:
    """Smooth seeded sinusoidal joint trajectory, (n_frames, n_joints) float64."""
    rng = np.random.default_rng(seed)
    amp = rng.uniform(0.3, 1.5, n_joints)
    freq = rng.uniform(0.05, 0.4, n_joints)
    ph = rng.uniform(-math.pi, math.pi, n_joints)
    t = np.arange(n_frames)[:, None] / fps
    return amp * np.sin(2 * math.pi * freq * t + ph)


def batch_dims(seed: int, n_maps: int = 64, lo: int = 64, hi: int = 192) -> np.ndarray:
    """(n_maps, 3) int32 grid extents, each axis uniform in {lo..hi}."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=(n_maps, 3)).astype(np.int32)
