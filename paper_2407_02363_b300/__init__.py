"""B300-native exact voxel distance maps for collision avoidance (arXiv 2407.02363).

The compute path lives in the C-ABI library `libvedt.so` (CUDA, sm_103a), declared in
include/vedt.h; `paper_2407_02363_b300.vedt` is its thin ctypes binding.  Importing
this package loads nothing: `synth` (seeded inputs) is usable without a GPU.
"""
__all__ = ["synth", "vedt"]
