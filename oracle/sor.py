"""Statistical outlier filter of the raw point cloud (Sec. III-A): a point is dropped when
its mean Euclidean distance to its k nearest neighbours lies more than `std_mul`
standard deviations above the mean of that quantity over the cloud.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy, brute force: every
distance to every other point, no spatial index.

The paper names the filter but gives neither k nor the multiplier; both are inputs.  The
arithmetic is fixed so that an independent implementation reaches the same keep
decision bit for bit:
  * valid points: all three coordinates finite; others are dropped and take no part;
  * d2(i, j) = ((xi - xj)^2 + (yi - yj)^2) + (zi - zj)^2 in float64 (differences of
    float32 values are exact in float64), self excluded (one zero distance for i);
  * k_i = min(k, m - 1) for m valid points; the k_i smallest d2 in ascending order,
    d_i = (sqrt(s_1) + sqrt(s_2) + ... + sqrt(s_k_i)) / k_i, summed left to right;
    d_i = 0 if k_i = 0;
  * the sums over the cloud are exact: S = sum floor(d_i * 2^80), Q = sum
    floor((d_i * d_i) * 2^80) as integers (any summation order gives the same S, Q);
  * s = float(S) * 2^-80, q = float(Q) * 2^-80, mean = s / m,
    var = (q - (s * s) / m) / (m - 1) (0 if m < 2, clamped at 0), std = sqrt(var),
    threshold = mean + std_mul * std;
  * keep_i = valid_i and d_i <= threshold.
"""
from __future__ import annotations

import math

import numpy as np

SCALE_BITS = 80


def fixed(x: float) -> int:
    """floor(x * 2^80) for x >= 0, exactly (the scaling by a power of two is exact)."""
    return int(math.floor(float(x) * 2.0 ** SCALE_BITS))


def mean_knn_distance(xyz: np.ndarray, k: int, block: int = 512):
    """d_i for every point (NaN for invalid points) and the valid mask."""
    p = np.asarray(xyz, dtype=np.float32).reshape(-1, 3)
    valid = np.isfinite(p).all(axis=1)
    q = p[valid].astype(np.float64)
    m = q.shape[0]
    d = np.full(p.shape[0], np.nan)
    if m == 0:
        return d, valid
    kk = min(k, m - 1)
    if kk == 0:
        d[valid] = 0.0
        return d, valid
    out = np.empty(m)
    for a in range(0, m, block):
        b = min(m, a + block)
        dx = q[a:b, 0:1] - q[None, :, 0]
        dy = q[a:b, 1:2] - q[None, :, 1]
        dz = q[a:b, 2:3] - q[None, :, 2]
        d2 = (dx * dx + dy * dy) + dz * dz
        d2[np.arange(b - a), np.arange(a, b)] = np.inf        # self
        near = np.partition(d2, kk - 1, axis=1)[:, :kk]
        near.sort(axis=1)
        r = np.sqrt(near)
        acc = np.zeros(b - a)
        for t in range(kk):                                    # left to right
            acc = acc + r[:, t]
        out[a:b] = acc / kk
    d[valid] = out
    return d, valid


def threshold(dv: np.ndarray, std_mul: float):
    """(mean, std, threshold) of the valid d_i by the exact sums above."""
    m = len(dv)
    S = sum(fixed(x) for x in dv)
    Q = sum(fixed(x * x) for x in dv)
    s = float(S) * 2.0 ** -SCALE_BITS
    q = float(Q) * 2.0 ** -SCALE_BITS
    mean = s / m
    var = (q - (s * s) / m) / (m - 1) if m > 1 else 0.0
    var = max(var, 0.0)
    std = math.sqrt(var)
    return mean, std, mean + float(std_mul) * std


def sor_filter(xyz: np.ndarray, k: int, std_mul: float):
    """keep (uint8 per point), d (float64 per point, NaN if invalid), (mean, std, thr)."""
    d, valid = mean_knn_distance(xyz, k)
    keep = np.zeros(len(d), np.uint8)
    if not valid.any():
        return keep, d, (math.nan, math.nan, math.nan)
    stats = threshold(d[valid], std_mul)
    keep[valid] = (d[valid] <= stats[2]).astype(np.uint8)
    return keep, d, stats
