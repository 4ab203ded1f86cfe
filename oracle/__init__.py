"""CPU oracle for the distance-map pipeline of arXiv 2407.02363.

TEST INFRASTRUCTURE ONLY.  Only the tests, `__graft_entry__.smoke()` and the
`cpu_baseline` / reference leg of `bench.py` may import this package.  It shares no
code with the CUDA library and never imports it.

Contents (each function cites the passage it follows):
  insert_points   Alg. 2 line 7 + robot-point removal, Sec. III-A   (C, fp32)
  insert_links    Alg. 2 lines 5-6, Sec. III-A / III-E               (C, fp32)
  edt             Alg. 1, Sec. III-C, separable, m1 = m2 = m3 = 1      (C, int64)
  edt_brute       the EDT's definition, Sec. III-C first paragraph     (C, int64)
  query_spheres   Eq. (dist), Alg. 2 line 10, Alg. 3 lines 3-4        (C, fp32)
  fk, sphere_centres   ForwardKinematics, Alg. 2 lines 5 and 8         (Python, fp64)
  mlp_*           learned surrogate reference (not in the paper)       (numpy, fp64)
  sor.sor_filter  statistical outlier filter of the raw cloud, Sec. III-A
                  (oracle/sor.py: numpy brute-force kNN, fp64, exact sums)
  logodds.update  Bayesian (log-odds) occupancy update, Sec. III-A (oracle/logodds.py)
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i32, i64, f32, u32 = ctypes.c_int, ctypes.c_int64, ctypes.c_float, ctypes.c_uint32
        L.oracle_insert_points.restype = i64
        L.oracle_insert_points.argtypes = [P, P, i32, i32, i32, f32, P, P, i64, P, i32]
        L.oracle_insert_links.restype = i64
        L.oracle_insert_links.argtypes = [P, i32, i32, i32, f32, P, i32, P, P, P, u32]
        L.oracle_edt.restype = None
        L.oracle_edt.argtypes = [P, i32, i32, i32, P, P, i32]
        L.oracle_edt_brute.restype = None
        L.oracle_edt_brute.argtypes = [P, i32, i32, i32, P, i64, P, P, i32]
        L.oracle_query.restype = None
        L.oracle_query.argtypes = [P, P, i32, i32, i32, f32, P, P, P, i32, P]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)))


SPHERE_DTYPE = np.dtype([("sqdist", "<i4"), ("idx", "<i4"), ("dist", "<f4"),
                         ("clearance", "<f4"), ("nearest", "<f4", (3,)), ("status", "<i4")])
STATUS_OK, STATUS_OUTSIDE, STATUS_EMPTY = 0, 1, 2


def insert_points(env, self_map, dims, vs, origin, xyz, T=None, filter_self=False):
    """Insert(Point_Cloud), Alg. 2 line 7; robot-point removal of Sec. III-A.
    env / self_map: uint8 (Z, Y, X), env modified in place.  Returns #points written."""
    X, Y, Z = dims
    assert env.dtype == np.uint8 and env.flags.c_contiguous and env.shape == (Z, Y, X)
    xyz = np.ascontiguousarray(xyz, dtype=np.float32)
    org = np.asarray(origin, dtype=np.float32)
    Tm = None if T is None else np.ascontiguousarray(T, dtype=np.float32).reshape(12)
    sm = None if self_map is None else np.ascontiguousarray(self_map, dtype=np.uint8)
    return lib().oracle_insert_points(_ptr(env), _ptr(sm), X, Y, Z, float(np.float32(vs)),
                                      _ptr(org), _ptr(xyz), xyz.shape[0], _ptr(Tm),
                                      1 if filter_self else 0)


def insert_links(self_map, dims, vs, origin, link_points, poses_f32, link_mask):
    """UpdateLinks + Insert(O_Lk), Alg. 2 lines 5-6.  link_points: list of (k_i, 3)
    float32 arrays in link frames; poses_f32: (n_links, 3, 4) float32."""
    X, Y, Z = dims
    assert self_map.dtype == np.uint8 and self_map.shape == (Z, Y, X)
    pts = np.ascontiguousarray(np.concatenate(link_points, axis=0), dtype=np.float32)
    offs = np.zeros(len(link_points) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([len(p) for p in link_points])
    poses = np.ascontiguousarray(poses_f32, dtype=np.float32).reshape(-1)
    org = np.asarray(origin, dtype=np.float32)
    return lib().oracle_insert_links(_ptr(self_map), X, Y, Z, float(np.float32(vs)), _ptr(org),
                                     len(link_points), _ptr(pts), _ptr(offs), _ptr(poses),
                                     int(link_mask))


def edt(occ, threads=None):
    """Exact EDT (Alg. 1 with m1 = m2 = m3 = 1).  occ: uint8 (Z, Y, X).
    Returns (sqdist int32, idx int32), both (Z, Y, X)."""
    occ = np.ascontiguousarray(occ, dtype=np.uint8)
    Z, Y, X = occ.shape
    sq = np.empty(occ.shape, dtype=np.int32)
    ix = np.empty(occ.shape, dtype=np.int32)
    lib().oracle_edt(_ptr(occ), X, Y, Z, _ptr(sq), _ptr(ix), threads or default_threads())
    return sq, ix


def edt_brute(occ, voxels=None, threads=None):
    """The EDT by definition at the given linear voxel indices (all voxels if None)."""
    occ = np.ascontiguousarray(occ, dtype=np.uint8)
    Z, Y, X = occ.shape
    q = np.arange(occ.size, dtype=np.int64) if voxels is None else np.ascontiguousarray(voxels, dtype=np.int64)
    sq = np.empty(q.shape[0], dtype=np.int32)
    ix = np.empty(q.shape[0], dtype=np.int32)
    lib().oracle_edt_brute(_ptr(occ), X, Y, Z, _ptr(q), q.shape[0], _ptr(sq), _ptr(ix),
                           threads or default_threads())
    return sq, ix


def query_spheres(sqdist, idx, dims, vs, origin, centres_f32, radii_f32):
    """ExtractClosestObstaclePose and x_ci = |O_i - C_i| at the voxel holding each
    sphere centre (Eq. (dist); Alg. 3 lines 3-4).  Returns a SPHERE_DTYPE array."""
    X, Y, Z = dims
    c = np.ascontiguousarray(centres_f32, dtype=np.float32).reshape(-1, 3)
    r = np.ascontiguousarray(radii_f32, dtype=np.float32).reshape(-1)
    out = np.zeros(c.shape[0], dtype=SPHERE_DTYPE)
    org = np.asarray(origin, dtype=np.float32)
    lib().oracle_query(_ptr(np.ascontiguousarray(sqdist, np.int32)),
                       _ptr(np.ascontiguousarray(idx, np.int32)), X, Y, Z,
                       float(np.float32(vs)), _ptr(org), _ptr(c), _ptr(r), c.shape[0], _ptr(out))
    return out


# ----------------------------------------------------------------------------------
# ForwardKinematics (Alg. 2 lines 5 and 8), fp64, products written out term by term
# ----------------------------------------------------------------------------------

def _compose(A, B):
    """A . B for 3x4 rigid transforms; each entry summed left to right."""
    C = [[0.0] * 4 for _ in range(3)]
    for i in range(3):
        for j in range(3):
            C[i][j] = (A[i][0] * B[0][j] + A[i][1] * B[1][j]) + A[i][2] * B[2][j]
        C[i][3] = ((A[i][0] * B[0][3] + A[i][1] * B[1][3]) + A[i][2] * B[2][3]) + A[i][3]
    return C


def _rz(q):
    c, s = math.cos(q), math.sin(q)
    return [[c, -s, 0.0, 0.0], [s, c, 0.0, 0.0], [0.0, 0.0, 1.0, 0.0]]


def fk(chain, q):
    """Poses of links 0..n in the world: T_0 = base, T_k = T_(k-1) . offset_k . Rz(q_k).
    Returns (n+1, 3, 4) float64."""
    T = [list(map(float, row)) for row in np.asarray(chain.base)]
    out = [T]
    for k in range(chain.n_joints):
        off = [list(map(float, row)) for row in np.asarray(chain.offsets[k])]
        T = _compose(_compose(T, off), _rz(float(q[k])))
        out.append(T)
    return np.array(out, dtype=np.float64)


def sphere_centres(chain, spheres, q):
    """World centres C_i of the bounding spheres (Alg. 2 line 8), fp64 then rounded to
    fp32: c_a = ((R_a0 l_0 + R_a1 l_1) + R_a2 l_2) + t_a."""
    P = fk(chain, q)
    out = np.empty((len(spheres.link), 3), dtype=np.float64)
    for i, (k, l) in enumerate(zip(spheres.link, spheres.local)):
        T = P[int(k)]
        for a in range(3):
            out[i, a] = ((T[a, 0] * l[0] + T[a, 1] * l[1]) + T[a, 2] * l[2]) + T[a, 3]
    return out.astype(np.float32)
