"""Autotuner for the batched EDT launch shapes.

The exact result never depends on the launch shape, only the time does.  The knobs are
those of vedt_batch_set_tuning: plain three-sweep launches versus one persistent launch,
and for the persistent launch the CTAs per SM and the pass-X rows per work item (the
role the band counts m1, m2, m3 of Alg. 1 play for PBA).  Each candidate is timed with
CUDA events on the batch's stream over a few repetitions of the EDT (after warm-up), the
fastest wins, and the winner is cached per (GPU name, grid-dimension signature) in a JSON
file so later runs skip the sweep.
"""
from __future__ import annotations

import hashlib
import json
import os
from dataclasses import asdict, dataclass

DEFAULT_CANDIDATES = (
    [(0, 0, 32)] +
    [(1, c, r) for c in (0, 2, 4, 8) for r in (8, 32, 128)]
)


@dataclass(frozen=True)
class Tuning:
    persistent: int
    ctas_per_sm: int
    rows_per_item: int

    def apply(self, batch):
        batch.set_tuning(self.ctas_per_sm, self.rows_per_item, self.persistent)


def cache_path() -> str:
    base = os.environ.get("VEDT_AUTOTUNE_CACHE")
    if base:
        return base
    root = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(root, "vedt", "autotune.json")


def signature(gpu_name: str, dims_list) -> str:
    """Cache key: the GPU and the multiset of grid extents in the batch."""
    dims = sorted(tuple(int(v) for v in d) for d in dims_list)
    h = hashlib.sha1(json.dumps(dims).encode()).hexdigest()[:16]
    return f"{gpu_name}|{len(dims)}|{h}"


def load_cache(path=None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store_cache(entries: dict, path=None):
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(entries, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def pick(times: dict) -> Tuning:
    """The candidate with the smallest time (ties: earliest in the sweep order)."""
    best = min(times.items(), key=lambda kv: kv[1])
    return best[0]


def time_candidate(batch, stream, tuning: Tuning, reps=5, warmup=2, op=None):
    """Median milliseconds of `op` (default: the batch EDT) under `tuning`."""
    import torch
    tuning.apply(batch)
    run = op or batch.compute_edt
    for _ in range(warmup):
        run()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    batch.check()
    ts.sort()
    return ts[len(ts) // 2]


def tune(batch, stream, dims_list, candidates=DEFAULT_CANDIDATES, reps=5, path=None, force=False, op=None):
    """Returns (best Tuning, {Tuning: ms}) and applies the best to `batch`.  A cached
    winner for the same GPU and dims is applied without timing unless force=True."""
    import torch
    gpu = torch.cuda.get_device_name()
    key = signature(gpu, dims_list)
    cache = load_cache(path)
    if not force and key in cache:
        t = Tuning(**cache[key]["tuning"])
        t.apply(batch)
        return t, {}
    times = {}
    for c in candidates:
        t = Tuning(*c)
        times[t] = time_candidate(batch, stream, t, reps=reps, op=op)
    best = pick(times)
    best.apply(batch)
    cache[key] = {"tuning": asdict(best), "ms": times[best],
                  "swept": {f"{t.persistent}/{t.ctas_per_sm}/{t.rows_per_item}": ms for t, ms in times.items()}}
    store_cache(cache, path)
    return best, times
