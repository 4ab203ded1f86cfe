"""Bayesian occupancy update of the environment map (Sec. III-A), integer log-odds form.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy.

The paper names a Bayesian per-voxel occupancy update but gives neither its model nor
its parameters.  Reading: each voxel keeps a log-odds value L (int8 range, 0 = unknown).  Every
frame, a voxel that at least one point of the frame maps to is a hit, every other voxel
a miss (no ray casting; the sensor sees the whole map):
    L <- clamp(L + l_hit, l_min, l_max)   on a hit
    L <- clamp(L - l_miss, l_min, l_max)  on a miss
and the voxel is occupied for the EDT iff L >= threshold.  With l_min = 0, l_miss = l_max and
0 < l_hit = threshold <= l_max this reduces to the one-hit rule of a map cleared every
frame (a miss takes L to 0, a hit to at least the threshold).
"""
from __future__ import annotations

import numpy as np


def update(L, hit, l_hit, l_miss, l_min, l_max, threshold):
    """One frame: returns (new L as int8, occupancy as uint8 0/1)."""
    L = np.asarray(L, np.int64)
    hit = np.asarray(hit) != 0
    step = np.where(hit, int(l_hit), -int(l_miss))
    Ln = np.clip(L + step, int(l_min), int(l_max))
    return Ln.astype(np.int8), (Ln >= int(threshold)).astype(np.uint8)
