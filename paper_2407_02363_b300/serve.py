"""Serving loop for control frames of mixed map sizes (continuous batching).

Each request is one control cycle of Alg. 2 (lines 4-10) for some map size: its point
cloud, joint state and sphere centres.  Maps stay resident on the device as slots keyed
by size; an arriving request takes an idle slot of its size, or a new slot if the free
device memory minus the slot's size stays above a headroom (and an optional byte budget
allows), or waits in the queue until one of those frees up.  Every slot has its own
stream, so frames admitted while others run overlap on the GPU; completion is polled
without blocking.  All compute runs in libvedt's kernels; this module only schedules.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import synth


@dataclass
class Request:
    rid: int
    dims: tuple
    cloud: object            # (n, 3) float32, page-locked torch tensor or numpy array
    q: np.ndarray            # joint angles
    centres: np.ndarray      # (m, 3) float32 sphere centres
    radii: np.ndarray        # (m,) float32
    arrival: float = 0.0     # seconds after the start of the run
    chain: object = None     # kinematic chain (vedt.Chain) of the robot in this map


@dataclass
class Done:
    rid: int
    dims: tuple
    arrival: float
    launched: float
    finished: float
    results: np.ndarray

    @property
    def latency(self):
        return self.finished - self.arrival


@dataclass
class Slot:
    dims: tuple
    map: object
    out: object = None
    m: int = 0
    req: Request = None
    launched: float = 0.0
    nbytes: int = 0
    frames: int = 0
    last_used: int = 0


@dataclass
class Server:
    """make_map(dims) -> map with frame_host_async / done (a vedt.Map on its own stream);
    free_fn() -> free device bytes; map_bytes(dims) -> bytes a slot allocates."""
    make_map: object
    free_fn: object
    map_bytes: object
    link_mask: int
    headroom: int = 1 << 30
    budget: int = None             # optional cap on slot bytes
    max_slots: int = 64
    alloc_out: object = None       # m -> page-locked result buffer
    view_out: object = None        # buffer -> SPHERE_DTYPE array (a copy)
    slots: list = field(default_factory=list)
    queue: collections.deque = field(default_factory=collections.deque)
    done: list = field(default_factory=list)
    release_map: object = None     # frees a slot's map (default: map.close())
    rejected_admissions: int = 0
    evictions: int = 0
    max_inflight: int = 0
    clock: int = 0

    def used_bytes(self):
        return sum(s.nbytes for s in self.slots)

    def _admissible(self, need):
        return (len(self.slots) < self.max_slots and self.free_fn() - need >= self.headroom and
                (self.budget is None or self.used_bytes() + need <= self.budget))

    def _slot_for(self, dims):
        for s in self.slots:
            if s.req is None and s.dims == dims:
                return s
        need = self.map_bytes(dims)
        have = any(s.dims == dims for s in self.slots)
        # make room by releasing idle slots of other sizes (least recently used first), but
        # only when this size has no slot at all: otherwise wait for one of its own slots,
        # since allocating and freeing device memory stalls the whole device
        while not self._admissible(need):
            idle = [s for s in self.slots if s.req is None and s.dims != dims]
            if have or not idle:
                self.rejected_admissions += 1
                return None
            victim = min(idle, key=lambda s: s.last_used)
            self.slots.remove(victim)
            (self.release_map or (lambda m: m.close()))(victim.map)
            self.evictions += 1
        s = Slot(dims=dims, map=self.make_map(dims), nbytes=need)
        self.slots.append(s)
        return s

    def submit(self, req: Request):
        self.queue.append(req)

    def poll(self, now: float):
        """Retire finished frames, then launch queued frames that can get a slot (in
        arrival order, skipping over frames whose size has no slot yet)."""
        for s in self.slots:
            if s.req is not None and s.map.done():
                r = s.req
                res = self.view_out(s.out)
                self.done.append(Done(r.rid, r.dims, r.arrival, s.launched, now, res))
                s.req = None
        waiting = collections.deque()
        while self.queue:
            r = self.queue.popleft()
            s = self._slot_for(r.dims)
            if s is None:
                waiting.append(r)
                continue
            if s.out is None or s.m != len(r.radii):
                s.out, s.m = self.alloc_out(len(r.radii)), len(r.radii)
            s.map.frame_host_async(r.cloud, r.chain, r.q, self.link_mask, r.centres, r.radii, s.out)
            s.req, s.launched = r, now
            s.frames += 1
            self.clock += 1
            s.last_used = self.clock
        self.queue = waiting
        self.max_inflight = max(self.max_inflight, sum(1 for s in self.slots if s.req is not None))

    def idle(self):
        return not self.queue and all(s.req is None for s in self.slots)

    def run(self, requests, realtime=True, poll_sleep=50e-6, timeout=120.0):
        """Feeds requests at their arrival times (or all at once) until all finish."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        t0 = time.perf_counter()
        while True:
            now = time.perf_counter() - t0
            while pending and (not realtime or pending[0].arrival <= now):
                r = pending.popleft()
                if not realtime:
                    r.arrival = now
                self.submit(r)
            self.poll(time.perf_counter() - t0)
            if not pending and self.idle():
                break
            if now > timeout:
                raise TimeoutError("serving run did not drain")
            if poll_sleep:
                time.sleep(poll_sleep)
        return self.done


def stats(done, voxels_of):
    lat = np.array([d.latency for d in done]) * 1e3
    span = max(d.finished for d in done) - min(d.arrival for d in done)
    vox = sum(voxels_of(d.dims) for d in done)
    by = collections.defaultdict(list)
    for d in done:
        by[d.dims[0]].append(d.latency * 1e3)
    return {"frames": len(done), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max()), "span_s": span, "gvoxel_s": vox / span / 1e9,
            "p50_ms_by_size": {str(k): float(np.percentile(v, 50)) for k, v in sorted(by.items())},
            "p99_ms_by_size": {str(k): float(np.percentile(v, 99)) for k, v in sorted(by.items())}}


# ------------------------------------------------------------------------------------
# synthetic request streams (seeded)
# ------------------------------------------------------------------------------------
def make_requests(seed, n, sizes=(128, 256, 512), rate_hz=120.0, voxel=0.01, points=(50_000, 1_000_000),
                  clouds_per_size=2, pin=True):
    """n requests: size uniform over `sizes` (cubic grids of `voxel` metres), a cloud of
    U[points] points from a depth-camera scene of that grid, a smooth joint trajectory,
    Poisson arrivals at `rate_hz` aggregate."""
    import torch

    from . import vedt as v
    rng = np.random.default_rng(seed)
    chain = {}
    clouds = {}
    for S in sizes:
        grid = synth.GridSpec((S, S, S), voxel)
        ch = synth.make_chain(seed, tuple(np.array(grid.extent) / 2))
        chain[S] = ch
        lst = []
        for c in range(clouds_per_size):
            npts = int(rng.integers(points[0], points[1] + 1))
            sc = synth.CameraScene(seed + 97 * S + c, grid, n_points=npts, resolution_scale=max(1.0, np.sqrt(npts / 250_000)))
            pts = sc.frame(c)
            t = torch.from_numpy(pts)
            lst.append(t.pin_memory() if pin else t)
        clouds[S] = lst
    spheres = synth.sphere_model(chain[sizes[0]])
    cchain = {S: v.make_chain(c) for S, c in chain.items()}
    traj = synth.joint_trajectory(seed, n)
    arr = np.cumsum(rng.exponential(1.0 / rate_hz, size=n))
    reqs = []
    for i in range(n):
        S = int(sizes[rng.integers(0, len(sizes))])
        cen = v.sphere_centres(cchain[S], spheres, traj[i])
        cl = clouds[S][int(rng.integers(0, len(clouds[S])))]
        reqs.append(Request(rid=i, dims=(S, S, S), cloud=cl, q=traj[i], centres=cen, radii=spheres.radius,
                            arrival=float(arr[i]), chain=cchain[S]))
    return reqs, chain, spheres


def gpu_server(chain_by_size, link_mask=0b111, voxel=0.01, headroom=4 << 30, budget=None, max_slots=16):
    """A Server whose slots are vedt maps on their own CUDA streams."""
    import torch

    from . import vedt as v

    def make_map(dims):
        S = dims[0]
        m = v.Map(dims, voxel, (0.0, 0.0, 0.0), stream=torch.cuda.Stream())
        m.register_links(synth.link_models(chain_by_size[S], voxel))
        return m

    def alloc_out(m):
        return torch.empty(2 * m * 32, dtype=torch.uint8).pin_memory()

    def view_out(buf):
        return buf.numpy().view(v.SPHERE_DTYPE).copy()

    return Server(make_map=make_map, free_fn=lambda: v.device_memory()[0], map_bytes=v.map_bytes,
                  link_mask=link_mask, headroom=headroom, budget=budget, max_slots=max_slots,
                  alloc_out=alloc_out, view_out=view_out)
