"""Builds libvedt.so (CUDA, sm_103a) in-tree from csrc/*.cu with plain nvcc.

    python -m paper_2407_02363_b300.build [--force] [--verbose] [--debug]

Each translation unit is compiled to an object with
`-gencode arch=compute_103a,code=sm_103a -O3 -lineinfo` (no fast-math: the insert and
query kernels rely on IEEE-rounded fp32), then linked into a shared library against the
shared CUDA runtime, so the process shares one runtime with PyTorch.  The translation
units compile in parallel.

`--debug` builds libvedt_debug.so instead, with -DVEDT_DEBUG_BOUNDS: the EDT passes check
every index they compute against its buffer and report a bad one through the map's error
word.  The binding loads it when VEDT_DEBUG_BOUNDS=1 is set in the environment.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libvedt.so")
DEBUG_LIB = os.path.join(HERE, "libvedt_debug.so")
BUILD = os.path.join(HERE, "_build")
INC = os.path.join(os.path.dirname(HERE), "include")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INC, "-I", CSRC,
                 "--expt-relaxed-constexpr", "-Xcompiler", "-ffp-contract=off"]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
            glob.glob(os.path.join(INC, "*.h")))


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    lib = DEBUG_LIB if debug else LIB
    if not force and up_to_date(lib):
        return lib
    bdir = BUILD + ("_debug" if debug else "")
    os.makedirs(bdir, exist_ok=True)
    flags = COMMON + (["-DVEDT_DEBUG_BOUNDS"] if debug else []) + (["-Xptxas", "-v"] if verbose else [])

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        r = subprocess.run([NVCC, "-c", src, "-o", obj] + flags, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    srcs = _sources()
    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, srcs))
    cmd = [NVCC, "-shared", "-o", lib] + objs + ARCH + ["-cudart", "shared",
                                                        "-Xlinker", "-rpath=/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv, debug="--debug" in sys.argv))
