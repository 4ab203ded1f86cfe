"""Autotuner for the EDT's band counts and launch shapes.

The exact result never depends on these knobs, only the time does (the m1 / m2 / m3 bands
of Alg. 1 are PBA's tunables, Sec. III-C; Tab. 2 compares band settings).

* Single maps and frames (`tune_map`): the bands per line of passes Y and Z
  (vedt_map_set_bands: 1, 2, 4 or 8 for grids with every dim <= 256; above, 4, 8 or the
  default, which takes eight bands for lines over 256 and four for the others) and
  the pass-Z tile shape (vedt_map_set_tile_z: 8 x 4 or 32 x 1 columns).
* Batches (`tune`): three plain launches (one per sweep) versus one persistent launch
  over a work queue, the bands per line and pass-Z tile shape of either, and for the
  persistent launch the CTAs per SM and the pass-X rows per work item
  (vedt_batch_set_tuning / _set_bands / _set_tile_z).

Each candidate is timed with CUDA events on the workload's stream over a few repetitions
(after warm-up); the fastest wins.  Winners are cached per (GPU name, grid-dimension
signature, workload kind) in a JSON file, so later runs, and maps or batches created
with `apply_cached_map` / `apply_cached`, take them without a sweep.
"""
from __future__ import annotations

import hashlib
import json
import os
from dataclasses import asdict, dataclass

BANDS_SMALL = (1, 2, 4, 8)    # grids with every dim <= 256
BANDS_LARGE = (0, 4, 8)       # 0: four or eight bands per pass by its line length
TILES_Z = (8, 32)             # pass-Z tile widths (8 x 4, 32 x 1 columns)


@dataclass(frozen=True)
class Tuning:
    persistent: int
    ctas_per_sm: int
    rows_per_item: int
    bands: int = 0
    tile_z: int = 0

    def apply(self, batch):
        batch.set_tile_z(self.tile_z)
        batch.set_tuning(self.ctas_per_sm, self.rows_per_item, self.persistent)
        batch.set_bands(self.bands)

    def label(self) -> str:
        return f"{self.persistent}/{self.ctas_per_sm}/{self.rows_per_item}/{self.bands}/{self.tile_z}"


@dataclass(frozen=True)
class MapTuning:
    bands: int
    tile_z: int = 0

    def apply(self, m):
        m.set_tile_z(self.tile_z)
        m.set_bands(self.bands)

    def label(self) -> str:
        return f"{self.bands}/{self.tile_z}"


def batch_candidates(large=False, bands=None, tiles=None):
    """Plain launches and persistent shapes, each at every admitted band count and pass-Z
    tile shape."""
    bs = bands or (BANDS_LARGE if large else BANDS_SMALL)
    out = []
    for tz in (tiles or TILES_Z):
        for b in bs:
            out.append((0, 0, 32, b, tz))
            out += [(1, c, r, b, tz) for c in (0, 4) for r in (16, 64)]
    return out


DEFAULT_CANDIDATES = batch_candidates()


def cache_path() -> str:
    base = os.environ.get("VEDT_AUTOTUNE_CACHE")
    if base:
        return base
    root = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(root, "vedt", "autotune.json")


def signature(gpu_name: str, dims_list, kind: str = "batch") -> str:
    """Cache key: the GPU, the workload kind and the multiset of grid extents."""
    dims = sorted(tuple(int(v) for v in d) for d in dims_list)
    h = hashlib.sha1(json.dumps(dims).encode()).hexdigest()[:16]
    return f"{gpu_name}|{kind}|{len(dims)}|{h}"


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


def pick(times: dict):
    """The candidate with the smallest time (ties: earliest in the sweep order)."""
    best = min(times.items(), key=lambda kv: kv[1])
    return best[0]


def _time(op, stream, reps, warmup):
    import torch
    for _ in range(warmup):
        op()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        op()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    ts.sort()
    return ts[len(ts) // 2]


def time_candidate(batch, stream, tuning: Tuning, reps=5, warmup=2, op=None):
    """Median milliseconds of `op` (default: the batch EDT) under `tuning`."""
    tuning.apply(batch)
    ms = _time(op or batch.compute_edt, stream, reps, warmup)
    batch.check()
    return ms


def _gpu():
    import torch
    return torch.cuda.get_device_name()


def _as_tuning(c):
    return c if isinstance(c, Tuning) else Tuning(*c)


def tune(batch, stream, dims_list, candidates=None, reps=5, path=None, force=False, op=None, kind="batch"):
    """Returns (best Tuning, {Tuning: ms}) and applies the best to `batch`.  A cached
    winner for the same GPU, dims and kind is applied without timing unless force=True."""
    large = any(max(int(v) for v in d) > 256 for d in dims_list)
    small = any(max(int(v) for v in d) <= 256 for d in dims_list)
    cands = [_as_tuning(c) for c in (candidates or batch_candidates(large, tiles=None if small else (0,)))]
    key = signature(_gpu(), dims_list, kind)
    cache = load_cache(path)
    if not force and key in cache:
        t = Tuning(**cache[key]["tuning"])
        t.apply(batch)
        return t, {}
    times = {t: time_candidate(batch, stream, t, reps=reps, op=op) for t in cands}
    best = pick(times)
    best.apply(batch)
    cache[key] = {"tuning": asdict(best), "ms": times[best], "swept": {t.label(): ms for t, ms in times.items()}}
    store_cache(cache, path)
    return best, times


def apply_cached(batch, dims_list, path=None, kind="batch"):
    """Applies a cached batch winner if there is one; returns it (or None)."""
    cache = load_cache(path)
    e = cache.get(signature(_gpu(), dims_list, kind))
    if not e:
        return None
    t = Tuning(**e["tuning"])
    t.apply(batch)
    return t


def map_candidates(dims):
    """Band counts admitted for a map of these dims."""
    return BANDS_LARGE if max(int(v) for v in dims) > 256 else BANDS_SMALL


def map_tunings(dims):
    """Every (bands, pass-Z tile shape) pair admitted for a map of these dims."""
    return [MapTuning(b, tz) for tz in TILES_Z for b in map_candidates(dims)]


def _map_entry(e) -> MapTuning:
    return MapTuning(**e["tuning"]) if "tuning" in e else MapTuning(int(e["bands"]))


def tune_map(m, stream, dims, op=None, candidates=None, reps=5, warmup=2, path=None, force=False, kind="edt"):
    """Bands per line and pass-Z tile shape for one map: times `op` (default: the EDT of
    both grids) under every candidate (MapTuning, or a band count for the default shape),
    applies and caches the fastest.  Returns (MapTuning, {MapTuning: ms})."""
    import paper_2407_02363_b300.vedt as v
    run = op or (lambda: m.compute_edt(v.MAP_BOTH))
    key = signature(_gpu(), [dims], kind)
    cache = load_cache(path)
    if not force and key in cache:
        t = _map_entry(cache[key])
        t.apply(m)
        return t, {}
    cands = [c if isinstance(c, MapTuning) else MapTuning(int(c)) for c in (candidates or map_tunings(dims))]
    times = {}
    for t in cands:
        t.apply(m)
        times[t] = _time(run, stream, reps, warmup)
    m.check()
    best = pick(times)
    best.apply(m)
    cache[key] = {"tuning": asdict(best), "ms": times[best], "swept": {t.label(): ms for t, ms in times.items()}}
    store_cache(cache, path)
    return best, times


def apply_cached_map(m, dims, path=None, kind="edt"):
    """Applies a map's cached winner of tune_map for these dims and kind on this GPU;
    returns it (a MapTuning) or None."""
    e = load_cache(path).get(signature(_gpu(), [dims], kind))
    if not e:
        return None
    t = _map_entry(e)
    t.apply(m)
    return t
