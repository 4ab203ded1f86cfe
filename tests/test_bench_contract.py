"""Host-side pieces of bench.py's report: the DRAM-traffic entry belongs to the kernel
source it was captured from, and the algorithmic bytes per launch are the design's
(1 B occupancy in, 8 B field out per voxel for the whole EDT; 10 B per voxel for pass Z)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_entry_matches_the_kernel_source():
    entry = bench.NCU_TRAFFIC["edt_z"]
    assert entry["src"] == bench.kernel_src_hash(), "pass-Z traffic was captured from other kernel source"
    n = 256 ** 3
    assert entry["alg_bytes_per_launch"] == n * 10
    # DRAM bytes at or below the algorithmic bytes (no wasted re-reads)
    assert 0 < entry["bytes"] <= entry["alg_bytes_per_launch"]


def test_code_hash_ignores_comments_and_blank_space():
    a = "int f(int x) { return x + 1; } // one\n/* two */\n"
    b = "int f(int x)\n{\n    return x + 1;   /* changed comment */\n}\n"
    assert bench.code_hash([a]) == bench.code_hash([b])
    assert bench.code_hash([a]) != bench.code_hash([a.replace("+ 1", "+ 2")])


def test_frame_bytes_per_kernel():
    n = 256 ** 3
    fb = lambda k: bench.frame_bytes(k, n, 300_000, 80_000)
    assert fb("edt_x") + fb("edt_y") + fb("edt_z") == 2 * n * (2 + 3 + 10)
    assert fb("edt_z") == 2 * n * 10
    assert fb("clear") == 2 * n
    assert fb("insert_points") == 300_000 * 12 and fb("insert_links") == 80_000 * 12
