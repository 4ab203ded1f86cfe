"""Command-line runs of single library calls on seeded synthetic inputs, for timing and
profiling one kernel family at a time:

    python -m paper_2407_02363_b300.run edt --dims 512 512 512 --voxel 0.02 --points 600000 --reps 3
    python -m paper_2407_02363_b300.run sor --points 300000 --k 50 --reps 3
    python -m paper_2407_02363_b300.run frame --dims 256 256 256 --voxel 0.01 --logodds --reps 3

`edt`: one map of the given dims, a depth-camera cloud (synth.CameraScene) inserted into
the environment grid, then `reps` EDTs of that grid.  `sor`: the statistical outlier filter
on a camera cloud of the given size.  `frame`: whole frames (vedt_frame: clear, cloud
insert, EDT of both grids; no arm), optionally with the log-odds occupancy of the
environment grid (`--logodds`, l_hit 9, l_miss 4, clamp [-20, 40], threshold 15).  Each
prints the device time per call (CUDA events).
"""
from __future__ import annotations

import argparse


def _main():
    import torch

    from . import build, synth
    from . import vedt as v
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=("edt", "sor", "frame"))
    ap.add_argument("--logodds", action="store_true")
    ap.add_argument("--dims", type=int, nargs=3, default=(256, 256, 256))
    ap.add_argument("--voxel", type=float, default=0.01)
    ap.add_argument("--points", type=int, default=300_000)
    ap.add_argument("--k", type=int, default=50)
    ap.add_argument("--std-mul", type=float, default=1.0)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=1234)
    a = ap.parse_args()
    build.build()
    grid = synth.GridSpec(tuple(a.dims), a.voxel)
    cloud = torch.from_numpy(synth.CameraScene(a.seed, grid, n_points=a.points).frame(0)).cuda()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if a.what == "frame":
        m = v.Map(grid.dims, grid.voxel_size, grid.origin)
        if a.logodds:
            m.set_logodds(True, l_hit=9, l_miss=4, l_min=-20, l_max=40, threshold=15)
        for _ in range(2):
            m.frame(cloud, cloud.shape[0], None, None, 0, None, None, 0, None)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(a.reps):
            m.frame(cloud, cloud.shape[0], None, None, 0, None, None, 0, None)
        e1.record()
        torch.cuda.synchronize()
        m.check()
        print(f"frame {tuple(a.dims)} logodds={a.logodds}: {e0.elapsed_time(e1) / a.reps:.4f} ms")
        m.close()
    elif a.what == "edt":
        m = v.Map(grid.dims, grid.voxel_size, grid.origin)
        m.clear(v.MAP_ENV)
        m.insert_pointcloud(cloud)
        m.compute_edt(v.MAP_ENV)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(a.reps):
            m.compute_edt(v.MAP_ENV)
        e1.record()
        torch.cuda.synchronize()
        m.check()
        print(f"edt {tuple(a.dims)}: {e0.elapsed_time(e1) / a.reps:.4f} ms")
        m.close()
    else:
        n = int(cloud.shape[0])
        f = v.OutlierFilter(n)
        keep = torch.empty(n, dtype=torch.uint8, device="cuda")
        f.filter(cloud, keep, k=a.k, std_mul=a.std_mul)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(a.reps):
            f.filter(cloud, keep, k=a.k, std_mul=a.std_mul)
        e1.record()
        torch.cuda.synchronize()
        (mean, std, thr), (valid, kept) = f.stats()
        print(f"sor {n} points k={a.k}: {e0.elapsed_time(e1) / a.reps:.4f} ms, kept {kept} of {valid}")
        f.close()


if __name__ == "__main__":
    _main()
