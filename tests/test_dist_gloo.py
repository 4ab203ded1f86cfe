"""Multi-rank host logic of bench.py on the CPU, with two gloo ranks (world_size 2) that
rendezvous on 127.0.0.1.

Under torchrun every rank runs its own independent maps and frames (weak scaling).  The
only collective is a max-reduction of timings and a barrier, never data.  The reference
arm (the CPU oracle) runs on rank 0 alone; other ranks exit at once."""
import os
import socket
import subprocess
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w, local = bench.dist_env()
    bench.dist_init(w, "gloo")
    bench.barrier(w)
    # each rank reports a different "elapsed time"; every rank must see the maximum
    got = bench.reduce_max(1.5 * (r + 1), w)
    bench.barrier(w)
    q.put((r, w, local, got))
    dist.destroy_process_group()


def test_two_gloo_ranks_share_only_the_max_of_timings():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 2, 0, 3.0), (1, 2, 1, 3.0)]


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(2.5, 1) == 2.5
    bench.barrier(1)   # no-op without a process group


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(_free_port()))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_ranks_draw_independent_frames():
    """Weak scaling: rank r's synthetic camera scene is seeded from the rank, so ranks do
    not process the same clouds."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2407_02363_b300 import synth
    g = synth.GridSpec(bench.DIMS, bench.VOXEL)
    a = synth.CameraScene(bench.SEED + 100 * 0, g, n_points=2000).frame(0)
    b = synth.CameraScene(bench.SEED + 100 * 1, g, n_points=2000).frame(0)
    assert a.shape == b.shape == (2000, 3)
    assert not np.array_equal(a, b)
