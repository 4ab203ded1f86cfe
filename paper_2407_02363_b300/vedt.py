"""Thin ctypes binding of libvedt.so (include/vedt.h).  Argument marshalling only:
every step of the pipeline runs in the library's CUDA kernels.  Importing this module
raises if the compiled library is missing; there is no CPU fallback.

Device buffers are passed as torch CUDA tensors (via data_ptr) or raw integers; streams
as torch.cuda.Stream objects or raw cudaStream_t integers.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# VEDT_DEBUG_BOUNDS=1 selects the bounds-checked build (python -m paper_2407_02363_b300.build --debug)
DEBUG_BOUNDS = os.environ.get("VEDT_DEBUG_BOUNDS") == "1"
LIB_PATH = os.path.join(_HERE, "libvedt_debug.so" if DEBUG_BOUNDS else "libvedt.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{os.path.basename(LIB_PATH)} not built at {LIB_PATH}; run "
                      f"`python -m paper_2407_02363_b300.build{' --debug' if DEBUG_BOUNDS else ''}`")

_lib = ctypes.CDLL(LIB_PATH)

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EBUSY, ENOTSUP = 0, -1, -2, -3, -4, -5, -6
MAP_ENV, MAP_SELF, MAP_BOTH = 1, 2, 3
SPHERE_OK, SPHERE_OUTSIDE, SPHERE_EMPTY = 0, 1, 2
MAX_DIM, MAX_LINKS, MAX_JOINTS = 1024, 16, 15
KERNELS = ("clear", "insert_links", "insert_points", "edt_x", "edt_y", "edt_z", "query", "occupancy")

SPHERE_DTYPE = np.dtype([("sqdist", "<i4"), ("idx", "<i4"), ("dist", "<f4"),
                         ("clearance", "<f4"), ("nearest", "<f4", (3,)), ("status", "<i4")])
assert SPHERE_DTYPE.itemsize == 32


class Chain(ctypes.Structure):
    _fields_ = [("n_joints", ctypes.c_int32), ("base", ctypes.c_double * 12),
                ("offset", (ctypes.c_double * 12) * MAX_JOINTS)]


class VedtError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


_P, _I32, _I64, _F32, _U32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_uint32
_sig = {
    "vedt_map_create": [_P, _F32, _P, _P, _P],
    "vedt_map_destroy": [_P],
    "vedt_map_set_stream": [_P, _P],
    "vedt_map_set_bands": [_P, _I32],
    "vedt_map_set_tile_z": [_P, _I32],
    "vedt_map_tile_z": [_P],
    "vedt_map_set_incremental": [_P, _I32],
    "vedt_map_set_logodds": [_P, _I32, _I32, _I32, _I32, _I32, _I32],
    "vedt_update_occupancy": [_P],
    "vedt_map_edt_recomputed": [_P, _I32, _P],
    "vedt_map_info": [_P, _P, _P, _P],
    "vedt_clear": [_P, _I32],
    "vedt_insert_pointcloud": [_P, _P, _I64, _P, _I32, _P],
    "vedt_insert_pointcloud_masked": [_P, _P, _I64, _P, _I32, _P, _P],
    "vedt_sor_create": [_I64, _P, _P],
    "vedt_sor_destroy": [_P],
    "vedt_sor_filter": [_P, _P, _I64, _I32, ctypes.c_double, _P],
    "vedt_sor_stats": [_P, _P, _P],
    "vedt_sor_mean_distances": [_P, _P],
    "vedt_register_links": [_P, _I32, _P, _P],
    "vedt_insert_links": [_P, _P, _U32],
    "vedt_fk": [_P, _P, _P],
    "vedt_insert_robot": [_P, _P, _P, _U32],
    "vedt_compute_edt": [_P, _I32],
    "vedt_query_spheres": [_P, _P, _P, _I32, _I32, _P],
    "vedt_query_spheres_dev": [_P, _P, _P, _I32, _I32, _P],
    "vedt_get_field": [_P, _I32, _P, _P],
    "vedt_get_occupancy": [_P, _I32, _P],
    "vedt_check": [_P],
    "vedt_set_timing": [_P, _I32],
    "vedt_kernel_times": [_P, _P, _P],
    "vedt_frame": [_P, _P, _I64, _P, _P, _P, _U32, _P, _P, _I32, _P],
    "vedt_frame_host": [_P, _P, _I64, _P, _P, _P, _U32, _P, _P, _I32, _P],
    "vedt_edt_noalloc": [_P, _I32, _I32, _I32, _P, _P, _P],
    "vedt_batch_create": [_P, _I32, _P, _P],
    "vedt_batch_destroy": [_P],
    "vedt_batch_set_tuning": [_P, _I32, _I32, _I32],
    "vedt_batch_set_bands": [_P, _I32],
    "vedt_batch_set_tile_z": [_P, _I32],
    "vedt_batch_tile_z": [_P],
    "vedt_batch_compute_edt": [_P],
    "vedt_batch_register_links": [_P, _I32, _P, _P],
    "vedt_batch_set_frame": [_P, _P, _P, _P, _U32, _P, _P, _I32, _P],
    "vedt_batch_run": [_P],
    "vedt_batch_capture": [_P],
    "vedt_batch_replay": [_P],
    "vedt_batch_check": [_P],
    "vedt_mlp_create": [_I32, _P, _P],
    "vedt_mlp_destroy": [_P],
    "vedt_mlp_set_params": [_P, _P, _I64],
    "vedt_mlp_get_params": [_P, _P, _I64],
    "vedt_mlp_get_state": [_P, _P, _P, _P, _I64, _P],
    "vedt_mlp_set_state": [_P, _P, _P, _P, _I64, _I64],
    "vedt_mlp_forward": [_P, _P, _I32, _P],
    "vedt_mlp_forward_layers": [_P, _P, _I32, _P],
    "vedt_mlp_grads": [_P, _P, _P, _P, _I32, _P, _I64, _P],
    "vedt_mlp_train_step": [_P, _P, _P, _P, _I32, _F32, _F32, _P],
    "vedt_mlp_check": [_P],
    "vedt_fk_batch": [_P, _P, _I64, _P],
    "vedt_sphere_centres": [_P, _P, _I32, _P, _P, _P],
    "vedt_sphere_centres_batch": [_P, _P, _I64, _I32, _P, _P, _P],
    "vedt_batch_set_grids": [_P, _I32],
    "vedt_frame_host_async": [_P, _P, _I64, _P, _P, _P, _U32, _P, _P, _I32, _P],
    "vedt_frame_done": [_P],
    "vedt_device_memory": [_P, _P],
    "vedt_selftest_wait": [_P, _U32],
}
for _n, _a in _sig.items():
    _f = getattr(_lib, _n)
    _f.argtypes = _a
    _f.restype = ctypes.c_int
_lib.vedt_status_string.argtypes = [ctypes.c_int]
_lib.vedt_status_string.restype = ctypes.c_char_p
_lib.vedt_version.restype = ctypes.c_char_p
_lib.vedt_mlp_num_params.restype = ctypes.c_int64
_lib.vedt_map_bytes.restype = ctypes.c_int64
_lib.vedt_map_bytes.argtypes = [ctypes.c_void_p]
_lib.vedt_mlp_num_params.argtypes = []


def status_string(s: int) -> str:
    return _lib.vedt_status_string(int(s)).decode()


def version() -> str:
    return _lib.vedt_version().decode()


def _chk(st, where):
    if st != OK:
        raise VedtError(st, where)


def _np_ptr(a):
    """Address of a numpy array's data for a C call.  Every caller binds the array to a name
    that outlives the call (the integer keeps no reference to it)."""
    return a.__array_interface__["data"][0]


def dev_ptr(x):
    """Device address of a torch tensor (or an int)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def stream_handle(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def edt_noalloc(occ_dev, dims, sqdist_dev, idx_dev, stream=None):
    """Exact EDT of one grid into caller-provided device buffers using the library's
    fixed static scratch (no device allocation; see vedt_edt_noalloc in include/vedt.h).
    occ_dev: contiguous CUDA uint8 tensor of X*Y*Z voxels; sqdist_dev, idx_dev: contiguous
    CUDA int32 tensors of at least X*Y*Z elements.  Returns once the fields are written."""
    import torch
    X, Y, Z = (int(v) for v in dims)
    n = X * Y * Z
    bufs = ((occ_dev, torch.uint8, "occupancy"), (sqdist_dev, torch.int32, "sqdist"), (idx_dev, torch.int32, "idx"))
    for t, dt, name in bufs:
        if not isinstance(t, torch.Tensor) or t.dtype != dt or not t.is_contiguous():
            raise ValueError(f"edt_noalloc: {name} must be a contiguous {dt} tensor")
        if t.numel() < n or (name == "occupancy" and t.numel() != n):
            raise ValueError(f"edt_noalloc: {name} holds {t.numel()} elements, the grid has {n}")
    for t, _, name in bufs:
        if not t.is_cuda:
            raise ValueError(f"edt_noalloc: {name} must be in device memory")
    _chk(_lib.vedt_edt_noalloc(dev_ptr(occ_dev), X, Y, Z, dev_ptr(sqdist_dev), dev_ptr(idx_dev),
                               stream_handle(stream)), "vedt_edt_noalloc")


def make_chain(chain) -> Chain:
    """Packs a synth.Chain-like object (base 3x4, offsets n x 3x4) into vedt_chain."""
    c = Chain()
    c.n_joints = chain.n_joints
    for i, v in enumerate(np.asarray(chain.base, dtype=np.float64).reshape(12)):
        c.base[i] = float(v)
    for k in range(chain.n_joints):
        for i, v in enumerate(np.asarray(chain.offsets[k], dtype=np.float64).reshape(12)):
            c.offset[k][i] = float(v)
    return c


def fk(chain, q) -> np.ndarray:
    c = chain if isinstance(chain, Chain) else make_chain(chain)
    qa = np.ascontiguousarray(q, dtype=np.float64)
    out = np.zeros((c.n_joints + 1, 3, 4), dtype=np.float64)
    _chk(_lib.vedt_fk(ctypes.byref(c), _np_ptr(qa), _np_ptr(out)), "vedt_fk")
    return out


def map_bytes(dims) -> int:
    """Device bytes a map of these dims allocates (admission control)."""
    d = np.ascontiguousarray(dims, dtype=np.int32)
    return int(_lib.vedt_map_bytes(_np_ptr(d)))


def device_memory():
    """(free, total) bytes of the current device."""
    f, t = ctypes.c_int64(), ctypes.c_int64()
    _chk(_lib.vedt_device_memory(ctypes.byref(f), ctypes.byref(t)), "vedt_device_memory")
    return int(f.value), int(t.value)


def fk_batch(chain, q) -> np.ndarray:
    """vedt_fk for many joint vectors: (n, n_joints + 1, 3, 4) float64 poses."""
    c = chain if isinstance(chain, Chain) else make_chain(chain)
    qa = np.ascontiguousarray(q, dtype=np.float64).reshape(-1, c.n_joints)
    out = np.zeros((qa.shape[0], c.n_joints + 1, 3, 4), dtype=np.float64)
    _chk(_lib.vedt_fk_batch(ctypes.byref(c), _np_ptr(qa), qa.shape[0], _np_ptr(out)), "vedt_fk_batch")
    return out


def sphere_centres(chain, spheres, q) -> np.ndarray:
    """C_i <- FK(q) (Alg. 2 line 8) through vedt_sphere_centres: (m, 3) float32 world
    centres of the spheres (`spheres.link`, `spheres.local` in link frames)."""
    c = chain if isinstance(chain, Chain) else make_chain(chain)
    qa = np.ascontiguousarray(q, dtype=np.float64)
    lk = np.ascontiguousarray(spheres.link, dtype=np.int32)
    lc = np.ascontiguousarray(spheres.local, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((lk.shape[0], 3), dtype=np.float32)
    _chk(_lib.vedt_sphere_centres(ctypes.byref(c), _np_ptr(qa), lk.shape[0], _np_ptr(lk), _np_ptr(lc),
                                  _np_ptr(out)), "vedt_sphere_centres")
    return out


class SphereCentres:
    """sphere_centres for one chain and sphere set, called once per control cycle: the
    sphere arrays and the (m, 3) result buffer are set up once and their addresses kept,
    so a call converts only the joint vector.  Each call returns the same buffer,
    overwritten; copy it to keep a cycle's centres."""

    def __init__(self, chain, spheres):
        self._chain = chain if isinstance(chain, Chain) else make_chain(chain)
        self._lk = np.ascontiguousarray(spheres.link, dtype=np.int32)
        self._lc = np.ascontiguousarray(spheres.local, dtype=np.float64).reshape(-1, 3)
        self.out = np.zeros((self._lk.shape[0], 3), dtype=np.float32)
        self._args = (ctypes.byref(self._chain), self._lk.shape[0], _np_ptr(self._lk), _np_ptr(self._lc),
                      _np_ptr(self.out))

    def __call__(self, q) -> np.ndarray:
        qa = np.ascontiguousarray(q, dtype=np.float64)
        cref, m, lk, lc, out = self._args
        _chk(_lib.vedt_sphere_centres(cref, _np_ptr(qa), m, lk, lc, out), "vedt_sphere_centres")
        return self.out


def sphere_centres_batch(chain, spheres, q) -> np.ndarray:
    """sphere_centres for many joint vectors: (n, m, 3) float32."""
    c = chain if isinstance(chain, Chain) else make_chain(chain)
    qa = np.ascontiguousarray(q, dtype=np.float64).reshape(-1, c.n_joints)
    lk = np.ascontiguousarray(spheres.link, dtype=np.int32)
    lc = np.ascontiguousarray(spheres.local, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((qa.shape[0], lk.shape[0], 3), dtype=np.float32)
    _chk(_lib.vedt_sphere_centres_batch(ctypes.byref(c), _np_ptr(qa), qa.shape[0], lk.shape[0], _np_ptr(lk),
                                        _np_ptr(lc), _np_ptr(out)), "vedt_sphere_centres_batch")
    return out


class Map:
    """Owns one vedt_map (environment M_I + self M_S grids and their distance fields)."""

    def __init__(self, dims, voxel_size, origin=(0.0, 0.0, 0.0), stream=None):
        d = np.ascontiguousarray(dims, dtype=np.int32)
        o = np.ascontiguousarray(origin, dtype=np.float32)
        h = ctypes.c_void_p()
        _chk(_lib.vedt_map_create(_np_ptr(d), float(voxel_size), _np_ptr(o), stream_handle(stream),
                                  ctypes.byref(h)), "vedt_map_create")
        self._h = h
        self.dims = tuple(int(v) for v in d)
        self.voxel_size = float(np.float32(voxel_size))
        self.origin = tuple(float(v) for v in o)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            _lib.vedt_map_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        _chk(_lib.vedt_map_set_stream(self._h, stream_handle(stream)), "vedt_map_set_stream")

    def set_bands(self, bands=0):
        """Bands per line of EDT passes Y and Z (0: default; 1/2/4/8 for dims <= 256, 4/8
        above)."""
        _chk(_lib.vedt_map_set_bands(self._h, int(bands)), "vedt_map_set_bands")

    def set_tile_z(self, cols_x=0):
        """Pass-Z tile shape: 8 (8 x 4 columns), 32 (32 x 1) or 0 (default); see
        vedt_map_set_tile_z.  Synchronises the map's streams."""
        _chk(_lib.vedt_map_set_tile_z(self._h, int(cols_x)), "vedt_map_set_tile_z")

    def tile_z(self):
        return int(_lib.vedt_map_tile_z(self._h))

    def set_logodds(self, on=True, l_hit=9, l_miss=4, l_min=-20, l_max=40, threshold=15):
        """Bayesian (log-odds) occupancy of the environment grid; see vedt_map_set_logodds."""
        _chk(_lib.vedt_map_set_logodds(self._h, 1 if on else 0, int(l_hit), int(l_miss), int(l_min), int(l_max),
                                       int(threshold)), "vedt_map_set_logodds")

    def update_occupancy(self):
        _chk(_lib.vedt_update_occupancy(self._h), "vedt_update_occupancy")

    def set_incremental(self, on=True):
        """Skip the EDT of a grid whose occupancy is unchanged since its last EDT."""
        _chk(_lib.vedt_map_set_incremental(self._h, 1 if on else 0), "vedt_map_set_incremental")

    def edt_recomputed(self, which=MAP_BOTH):
        """Per selected grid (env first): did the last compute_edt recompute it?"""
        out = np.zeros(2, dtype=np.int32)
        _chk(_lib.vedt_map_edt_recomputed(self._h, int(which), _np_ptr(out)), "vedt_map_edt_recomputed")
        return [bool(v) for v in out[: 2 if which == MAP_BOTH else 1]]

    def clear(self, which=MAP_BOTH):
        _chk(_lib.vedt_clear(self._h, which), "vedt_clear")

    def insert_pointcloud(self, xyz_dev, n=None, T_world_sensor=None, filter_self=False, counts_dev=None):
        n = int(xyz_dev.shape[0]) if n is None else int(n)
        T = None
        if T_world_sensor is not None:
            T = np.ascontiguousarray(T_world_sensor, dtype=np.float32).reshape(12)
        _chk(_lib.vedt_insert_pointcloud(self._h, dev_ptr(xyz_dev), n, None if T is None else _np_ptr(T),
                                         1 if filter_self else 0, dev_ptr(counts_dev)),
             "vedt_insert_pointcloud")

    def insert_pointcloud_masked(self, xyz_dev, keep_dev, n=None, T_world_sensor=None, filter_self=False,
                                 counts_dev=None):
        n = int(xyz_dev.shape[0]) if n is None else int(n)
        T = None
        if T_world_sensor is not None:
            T = np.ascontiguousarray(T_world_sensor, dtype=np.float32).reshape(12)
        _chk(_lib.vedt_insert_pointcloud_masked(self._h, dev_ptr(xyz_dev), n, None if T is None else _np_ptr(T),
                                                1 if filter_self else 0, dev_ptr(keep_dev), dev_ptr(counts_dev)),
             "vedt_insert_pointcloud_masked")

    def register_links(self, link_points):
        arrs = [np.ascontiguousarray(p, dtype=np.float32).reshape(-1, 3) for p in link_points]
        ptrs = (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
        nv = np.array([a.shape[0] for a in arrs], dtype=np.int64)
        _chk(_lib.vedt_register_links(self._h, len(arrs), ptrs, _np_ptr(nv)), "vedt_register_links")
        self._links = arrs

    def insert_links(self, poses_f32, link_mask):
        P = np.ascontiguousarray(poses_f32, dtype=np.float32).reshape(-1)
        _chk(_lib.vedt_insert_links(self._h, _np_ptr(P), int(link_mask)), "vedt_insert_links")

    def insert_robot(self, chain, q, link_mask):
        c = chain if isinstance(chain, Chain) else make_chain(chain)
        qa = np.ascontiguousarray(q, dtype=np.float64)
        _chk(_lib.vedt_insert_robot(self._h, ctypes.byref(c), _np_ptr(qa), int(link_mask)), "vedt_insert_robot")

    def compute_edt(self, which=MAP_BOTH):
        _chk(_lib.vedt_compute_edt(self._h, which), "vedt_compute_edt")

    def query_spheres(self, centres, radii, which=MAP_BOTH) -> np.ndarray:
        c = np.ascontiguousarray(centres, dtype=np.float32).reshape(-1, 3)
        r = np.ascontiguousarray(radii, dtype=np.float32).reshape(-1)
        ng = 2 if which == MAP_BOTH else 1
        out = np.zeros(c.shape[0] * ng, dtype=SPHERE_DTYPE)
        _chk(_lib.vedt_query_spheres(self._h, _np_ptr(c), _np_ptr(r), c.shape[0], which, _np_ptr(out)),
             "vedt_query_spheres")
        return out

    def query_spheres_dev(self, centres_dev, radii_dev, m, which, out_dev):
        _chk(_lib.vedt_query_spheres_dev(self._h, dev_ptr(centres_dev), dev_ptr(radii_dev), int(m), which,
                                         dev_ptr(out_dev)), "vedt_query_spheres_dev")

    def frame(self, xyz_dev, n, chain, q, link_mask, centres_dev, radii_dev, m, out_dev, T_world_sensor=None):
        """One control cycle on device buffers (vedt_frame), asynchronous."""
        T = None if T_world_sensor is None else np.ascontiguousarray(T_world_sensor, np.float32).reshape(12)
        qa = None if q is None else np.ascontiguousarray(q, dtype=np.float64)
        _chk(_lib.vedt_frame(self._h, dev_ptr(xyz_dev), int(n), None if T is None else _np_ptr(T),
                             None if chain is None else ctypes.byref(chain), None if qa is None else _np_ptr(qa),
                             int(link_mask), dev_ptr(centres_dev), dev_ptr(radii_dev), int(m), dev_ptr(out_dev)),
             "vedt_frame")

    def frame_host(self, xyz_host, chain, q, link_mask, centres, radii, out=None, T_world_sensor=None):
        """One control cycle from host buffers (vedt_frame_host); returns the 2m results."""
        x = np.ascontiguousarray(xyz_host, dtype=np.float32).reshape(-1, 3) if not hasattr(xyz_host, "data_ptr") \
            else xyz_host
        n = int(x.shape[0])
        xp = _np_ptr(x) if isinstance(x, np.ndarray) else x.data_ptr()
        c = np.ascontiguousarray(centres, dtype=np.float32).reshape(-1, 3)
        r = np.ascontiguousarray(radii, dtype=np.float32).reshape(-1)
        if out is None:
            out = np.zeros(2 * c.shape[0], dtype=SPHERE_DTYPE)
        T = None if T_world_sensor is None else np.ascontiguousarray(T_world_sensor, np.float32).reshape(12)
        qa = np.ascontiguousarray(q, dtype=np.float64)
        _chk(_lib.vedt_frame_host(self._h, xp, n, None if T is None else _np_ptr(T),
                                  None if chain is None else ctypes.byref(chain), _np_ptr(qa), int(link_mask),
                                  _np_ptr(c), _np_ptr(r), c.shape[0], _np_ptr(out)), "vedt_frame_host")
        return out

    def frame_host_async(self, xyz_host, chain, q, link_mask, centres, radii, out, T_world_sensor=None):
        """Queues one control cycle from host buffers (vedt_frame_host_async); `xyz_host`
        and `out` (a SPHERE_DTYPE array of 2m, or a pinned torch uint8 tensor) must stay
        alive until done() is true."""
        if hasattr(xyz_host, "data_ptr"):
            n, xp = int(xyz_host.shape[0]), xyz_host.data_ptr()
        else:
            n, xp = int(xyz_host.shape[0]), _np_ptr(xyz_host)
        c = np.ascontiguousarray(centres, dtype=np.float32).reshape(-1, 3)
        r = np.ascontiguousarray(radii, dtype=np.float32).reshape(-1)
        op = out.data_ptr() if hasattr(out, "data_ptr") else _np_ptr(out)
        T = None if T_world_sensor is None else np.ascontiguousarray(T_world_sensor, np.float32).reshape(12)
        qa = np.ascontiguousarray(q, dtype=np.float64)
        _chk(_lib.vedt_frame_host_async(self._h, xp, n, None if T is None else _np_ptr(T),
                                        None if chain is None else ctypes.byref(chain), _np_ptr(qa), int(link_mask),
                                        _np_ptr(c), _np_ptr(r), c.shape[0], op), "vedt_frame_host_async")

    def done(self):
        """True once every queued asynchronous frame has completed (raises on failure)."""
        st = _lib.vedt_frame_done(self._h)
        if st == EBUSY:
            return False
        _chk(st, "vedt_frame_done")
        return True

    def field_ptrs(self, which):
        sq, ix = ctypes.c_void_p(), ctypes.c_void_p()
        _chk(_lib.vedt_get_field(self._h, which, ctypes.byref(sq), ctypes.byref(ix)), "vedt_get_field")
        return sq.value, ix.value

    def occupancy_ptr(self, which):
        p = ctypes.c_void_p()
        _chk(_lib.vedt_get_occupancy(self._h, which, ctypes.byref(p)), "vedt_get_occupancy")
        return p.value

    def check(self):
        _chk(_lib.vedt_check(self._h), "vedt_check")

    def set_timing(self, enable=True):
        _chk(_lib.vedt_set_timing(self._h, 1 if enable else 0), "vedt_set_timing")

    def kernel_times(self):
        ms = np.zeros(len(KERNELS), dtype=np.float64)
        cnt = np.zeros(len(KERNELS), dtype=np.int64)
        _chk(_lib.vedt_kernel_times(self._h, _np_ptr(ms), _np_ptr(cnt)), "vedt_kernel_times")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNELS)}

    # --- torch views of device buffers ---
    def field_view(self, which):
        """Borrowed zero-copy (sqdist, idx) torch views (Z, Y, X) of the selected field."""
        X, Y, Z = self.dims
        sq, ix = self.field_ptrs(which)
        return device_view(sq, (Z, Y, X), "<i4"), device_view(ix, (Z, Y, X), "<i4")

    def field(self, which):
        """(sqdist, idx) as new torch int32 CUDA tensors of shape (Z, Y, X)."""
        self.check()
        sq, ix = self.field_view(which)
        return sq.clone(), ix.clone()

    def occupancy_view(self, which):
        X, Y, Z = self.dims
        return device_view(self.occupancy_ptr(which), (Z, Y, X), "|u1")

    def occupancy(self, which):
        self.check()
        return self.occupancy_view(which).clone()

    def upload_occupancy(self, which, occ):
        """Copies a uint8 (Z, Y, X) array (numpy or torch) into the selected grid."""
        import torch
        self.check()
        dst = self.occupancy_view(which)
        src = torch.as_tensor(np.ascontiguousarray(occ, dtype=np.uint8)) if isinstance(occ, np.ndarray) else occ
        dst.copy_(src.reshape(dst.shape))
        torch.cuda.synchronize()


class OutlierFilter:
    """Statistical outlier filter of a raw cloud (vedt_sor_*): keep flags per point."""

    def __init__(self, max_points, stream=None):
        h = ctypes.c_void_p()
        _chk(_lib.vedt_sor_create(int(max_points), stream_handle(stream), ctypes.byref(h)), "vedt_sor_create")
        self._h = h

    def close(self):
        if self._h:
            _lib.vedt_sor_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def filter(self, xyz_dev, keep_dev, k=50, std_mul=1.0, n=None):
        n = int(xyz_dev.shape[0]) if n is None else int(n)
        _chk(_lib.vedt_sor_filter(self._h, dev_ptr(xyz_dev), n, int(k), float(std_mul), dev_ptr(keep_dev)),
             "vedt_sor_filter")

    def stats(self):
        """((mean, std, threshold), (valid points, kept points)) of the last call."""
        st = np.zeros(3, np.float64)
        ct = np.zeros(2, np.int64)
        _chk(_lib.vedt_sor_stats(self._h, _np_ptr(st), _np_ptr(ct)), "vedt_sor_stats")
        return tuple(float(v) for v in st), tuple(int(v) for v in ct)

    def mean_distances(self, n):
        """The last call's d_i as a borrowed float64 device view of n entries."""
        p = ctypes.c_void_p()
        _chk(_lib.vedt_sor_mean_distances(self._h, ctypes.byref(p)), "vedt_sor_mean_distances")
        return device_view(p.value, (int(n),), "<f8")


class Batch:
    """Many maps processed together (vedt_batch_*): batched pipeline launches, one
    persistent EDT launch, optional CUDA-graph capture."""

    def __init__(self, maps, stream=None):
        self.maps = list(maps)
        arr = (ctypes.c_void_p * len(self.maps))(*[m.handle.value for m in self.maps])
        h = ctypes.c_void_p()
        _chk(_lib.vedt_batch_create(arr, len(self.maps), stream_handle(stream), ctypes.byref(h)), "vedt_batch_create")
        self._h = h

    def close(self):
        if self._h:
            _lib.vedt_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tuning(self, ctas_per_sm=0, rows_per_item=32, persistent=True):
        _chk(_lib.vedt_batch_set_tuning(self._h, int(ctas_per_sm), int(rows_per_item), 1 if persistent else 0),
             "vedt_batch_set_tuning")

    def set_bands(self, bands=0):
        _chk(_lib.vedt_batch_set_bands(self._h, int(bands)), "vedt_batch_set_bands")

    def set_tile_z(self, cols_x=0):
        _chk(_lib.vedt_batch_set_tile_z(self._h, int(cols_x)), "vedt_batch_set_tile_z")

    def tile_z(self):
        return int(_lib.vedt_batch_tile_z(self._h))

    def compute_edt(self):
        _chk(_lib.vedt_batch_compute_edt(self._h), "vedt_batch_compute_edt")

    def set_grids(self, which):
        _chk(_lib.vedt_batch_set_grids(self._h, int(which)), "vedt_batch_set_grids")

    def register_links(self, link_points):
        arrs = [np.ascontiguousarray(p, dtype=np.float32).reshape(-1, 3) for p in link_points]
        ptrs = (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
        nv = np.array([a.shape[0] for a in arrs], dtype=np.int64)
        _chk(_lib.vedt_batch_register_links(self._h, len(arrs), ptrs, _np_ptr(nv)), "vedt_batch_register_links")
        self._links = arrs

    def set_frame(self, xyz_dev, offsets, poses_f32, link_mask, centres_dev, radii_dev, m, out_dev):
        offs = np.ascontiguousarray(offsets, dtype=np.int64)
        P = np.ascontiguousarray(poses_f32, dtype=np.float32)
        _chk(_lib.vedt_batch_set_frame(self._h, dev_ptr(xyz_dev), _np_ptr(offs), _np_ptr(P), int(link_mask),
                                       dev_ptr(centres_dev), dev_ptr(radii_dev), int(m), dev_ptr(out_dev)),
             "vedt_batch_set_frame")

    def run(self):
        _chk(_lib.vedt_batch_run(self._h), "vedt_batch_run")

    def capture(self):
        _chk(_lib.vedt_batch_capture(self._h), "vedt_batch_capture")

    def replay(self):
        _chk(_lib.vedt_batch_replay(self._h), "vedt_batch_replay")

    def check(self):
        _chk(_lib.vedt_batch_check(self._h), "vedt_batch_check")


class MLP:
    """The learned self-distance surrogate (vedt_mlp_*): forward, gradients and AdamW
    steps in the library's tensor-core kernels."""

    def __init__(self, batch_capacity, stream=None):
        h = ctypes.c_void_p()
        _chk(_lib.vedt_mlp_create(int(batch_capacity), stream_handle(stream), ctypes.byref(h)), "vedt_mlp_create")
        self._h = h
        self.cap = int(batch_capacity)
        self.n_params = int(_lib.vedt_mlp_num_params())

    def close(self):
        if self._h:
            _lib.vedt_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        _chk(_lib.vedt_mlp_set_params(self._h, _np_ptr(p), p.size), "vedt_mlp_set_params")

    def get_params(self):
        p = np.zeros(self.n_params, dtype=np.float32)
        _chk(_lib.vedt_mlp_get_params(self._h, _np_ptr(p), p.size), "vedt_mlp_get_params")
        return p

    def get_state(self):
        """(params, AdamW first moments, second moments, step) for a checkpoint."""
        p, m1, m2 = (np.zeros(self.n_params, dtype=np.float32) for _ in range(3))
        step = ctypes.c_int64()
        _chk(_lib.vedt_mlp_get_state(self._h, _np_ptr(p), _np_ptr(m1), _np_ptr(m2), p.size, ctypes.byref(step)),
             "vedt_mlp_get_state")
        return p, m1, m2, int(step.value)

    def set_state(self, params, m1, m2, step):
        p, a, b = (np.ascontiguousarray(x, dtype=np.float32) for x in (params, m1, m2))
        _chk(_lib.vedt_mlp_set_state(self._h, _np_ptr(p), _np_ptr(a), _np_ptr(b), p.size, int(step)),
             "vedt_mlp_set_state")

    def save(self, path):
        """Writes the training state to an .npz file (parameters, moments, step)."""
        p, m1, m2, step = self.get_state()
        np.savez(path, params=p, m1=m1, m2=m2, step=np.int64(step))

    def load(self, path):
        """Restores a state written by save(); training continues from its step."""
        with np.load(path) as z:
            self.set_state(z["params"], z["m1"], z["m2"], int(z["step"]))

    def forward(self, q_dev, out_dev, B=None):
        B = int(q_dev.shape[0]) if B is None else int(B)
        _chk(_lib.vedt_mlp_forward(self._h, dev_ptr(q_dev), B, dev_ptr(out_dev)), "vedt_mlp_forward")

    def forward_layers(self, q_dev, out_dev, B=None):
        B = int(q_dev.shape[0]) if B is None else int(B)
        _chk(_lib.vedt_mlp_forward_layers(self._h, dev_ptr(q_dev), B, dev_ptr(out_dev)), "vedt_mlp_forward_layers")

    def grads(self, q_dev, y_dev, mask_dev=None, B=None):
        B = int(q_dev.shape[0]) if B is None else int(B)
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = ctypes.c_float()
        _chk(_lib.vedt_mlp_grads(self._h, dev_ptr(q_dev), dev_ptr(y_dev), dev_ptr(mask_dev), B, _np_ptr(g), g.size,
                                 ctypes.byref(loss)), "vedt_mlp_grads")
        return float(loss.value), g

    def train_step(self, q_dev, y_dev, mask_dev=None, lr=1e-3, wd=0.0, loss_sums_dev=None, B=None):
        B = int(q_dev.shape[0]) if B is None else int(B)
        _chk(_lib.vedt_mlp_train_step(self._h, dev_ptr(q_dev), dev_ptr(y_dev), dev_ptr(mask_dev), B, float(lr),
                                      float(wd), dev_ptr(loss_sums_dev)), "vedt_mlp_train_step")

    def check(self):
        _chk(_lib.vedt_mlp_check(self._h), "vedt_mlp_check")


class _CudaArray:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def device_view(ptr, shape, typestr):
    """Zero-copy torch CUDA tensor over library-owned device memory (borrowed)."""
    import torch
    return torch.as_tensor(_CudaArray(ptr, shape, typestr), device="cuda")


def exported_symbols():
    """Names declared in include/vedt.h that this library must export."""
    return list(_sig) + ["vedt_status_string", "vedt_version"]
