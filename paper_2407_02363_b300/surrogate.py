"""Learned surrogate for the self-collision distances (not in the paper).

The exact path (Sec. III-E: insert the self-obstacle links O_L into the self map, exact
EDT, read x_si of Eq. (selftaskvar) at the sphere centres) labels joint configurations;
a BF16 MLP trained on those labels by the library's tensor-core kernels predicts the 24
per-sphere distances directly from the joint angles.  At query time every configuration
whose predicted (unmasked) distance falls below a safety margin is recomputed by the
exact path, so near-collision decisions always come from the exact EDT.

All compute runs in libvedt (CUDA); this module only schedules it.
"""
from __future__ import annotations

import math
import os
import time
from dataclasses import dataclass

import numpy as np

from . import synth
from . import vedt as v

SELF_MASK = 0b111        # static body + links 1-2 form the self-collision obstacle O_L
# Distances are learned and compared up to this value: beyond it a sphere is far from
# every self obstacle, the collision-avoidance task is inactive (its activation only
# starts within the sphere radius plus a 2 cm buffer) and the exact value is irrelevant.
DIST_CLIP = 0.35


class ExactSelfDistance:
    """Exact per-sphere self distances for batches of joint configurations: one 128^3 /
    2 cm self map per configuration, n_maps configurations per CUDA-graph replay."""

    def __init__(self, chain, spheres, dims=(128, 128, 128), voxel_size=0.02, n_maps=256, self_mask=SELF_MASK,
                 stream=None):
        import torch
        self.torch = torch
        self.chain, self.spheres = chain, spheres
        self.cchain = v.make_chain(chain)
        self.n_maps, self.mask = n_maps, self_mask
        self.stream = stream or torch.cuda.Stream()
        self.maps = [v.Map(dims, voxel_size, (0.0, 0.0, 0.0), stream=self.stream) for _ in range(n_maps)]
        self.batch = v.Batch(self.maps, stream=self.stream)
        self.batch.set_grids(v.MAP_SELF)
        links = synth.link_models(chain, voxel_size)
        self.n_links = len(links)
        self.batch.register_links(links)
        m = len(spheres.radius)
        self.m = m
        self.cen = torch.zeros((n_maps, m, 3), dtype=torch.float32, device="cuda")
        self.radii = torch.from_numpy(spheres.radius.astype(np.float32)).cuda()
        self.out = torch.zeros(n_maps * 2 * m * 32, dtype=torch.uint8, device="cuda")
        self.offs = np.zeros(n_maps + 1, dtype=np.int64)
        self.poses = np.zeros((n_maps, self.n_links, 3, 4), dtype=np.float32)
        self.batch.set_frame(None, self.offs, self.poses, self_mask, self.cen, self.radii, m, self.out)
        self.batch.capture()

    def __call__(self, q):
        """(N, 7) joint angles -> (dist (N, m) float32 metres, status (N, m) int32)."""
        q = np.asarray(q, dtype=np.float64)
        N = q.shape[0]
        dist = np.empty((N, self.m), np.float32)
        stat = np.empty((N, self.m), np.int32)
        for s in range(0, N, self.n_maps):
            qc = q[s:s + self.n_maps]
            n = qc.shape[0]
            if n < self.n_maps:
                qc = np.concatenate([qc, np.repeat(qc[-1:], self.n_maps - n, axis=0)])
            P = v.fk_batch(self.cchain, qc)
            self.poses[:] = P[:, : self.n_links].astype(np.float32)
            self.cen.copy_(self.torch.from_numpy(v.sphere_centres_batch(self.cchain, self.spheres, qc)))
            self.batch.set_frame(None, self.offs, self.poses, self.mask, self.cen, self.radii, self.m, self.out)
            self.batch.replay()
            self.batch.check()
            res = self.out.cpu().numpy().view(v.SPHERE_DTYPE).reshape(self.n_maps, 2, self.m)[:n, 1]
            dist[s:s + n] = res["dist"]
            stat[s:s + n] = res["status"]
        return dist, stat

    def valid_mask(self, stat):
        """Spheres that count: inside the grid, on a link not adjacent to O_L."""
        return (stat == v.SPHERE_OK) & ~self.spheres.acm[None, :]

    def close(self):
        self.batch.close()
        for m in self.maps:
            m.close()


def clip(d):
    return np.minimum(d, DIST_CLIP)


@dataclass
class EvalResult:
    max_err_mm: float
    p99_err_mm: float
    mean_err_mm: float
    fallback_rate: float
    missed_rate: float
    margin_m: float
    n: int


def evaluate(pred, exact, valid, margin=0.05):
    """Errors (mm) over valid entries; a configuration falls back to the exact path if any
    valid predicted distance is below its sphere's margin (`margin`: one value for every
    sphere, or one per sphere); it is missed if it does not fall back but some valid exact
    distance is below 5 cm.  margin_m reports the largest margin."""
    err = np.abs(pred - exact)[valid] * 1000.0
    big = np.where(valid, pred, np.inf)
    fallback = (big < np.asarray(margin)).any(axis=1)
    near = (np.where(valid, exact, np.inf) < 0.05).any(axis=1)
    missed = near & ~fallback
    return EvalResult(max_err_mm=float(err.max()) if err.size else 0.0,
                      p99_err_mm=float(np.percentile(err, 99)) if err.size else 0.0,
                      mean_err_mm=float(err.mean()) if err.size else 0.0,
                      fallback_rate=float(fallback.mean()), missed_rate=float(missed.mean()),
                      margin_m=float(np.max(margin)), n=int(pred.shape[0]))


def sphere_margins(pred, exact, valid, base=0.05):
    """Per-sphere safety margins from a calibration set: base + the largest |error| of that
    sphere over its valid entries (base alone for a sphere with none).  If every error of a
    sphere stays within its calibration maximum, a prediction at or above the margin means
    an exact distance of at least `base`: pred < exact + e_max < base + e_max whenever
    exact < base.  A single margin (base + the largest error of any sphere) is the special
    case of the worst sphere; spheres whose network is more accurate fall back less."""
    err = np.where(valid, np.abs(pred - exact), 0.0)
    return base + err.max(axis=0)


def train(net, q, y, mask, steps, batch=8192, lr=2e-3, wd=1e-4, seed=0, log_every=0):
    """AdamW with cosine decay over `steps` minibatches drawn from device tensors q, y,
    mask (N x 7, N x 24, N x 24).  Returns the loss history (every log_every steps)."""
    import torch
    N = q.shape[0]
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    sums = torch.zeros(2, device="cuda")
    hist = []
    perm = torch.randperm(N, device="cuda", generator=g)
    pos = 0
    for it in range(steps):
        if pos + batch > N:
            perm = torch.randperm(N, device="cuda", generator=g)
            pos = 0
        idx = perm[pos:pos + batch]
        pos += batch
        qb, yb, mb = q[idx].contiguous(), y[idx].contiguous(), mask[idx].contiguous()
        cur = lr * 0.5 * (1 + math.cos(math.pi * it / max(1, steps)))
        net.train_step(qb, yb, mb, lr=cur, wd=wd, loss_sums_dev=sums)
        if log_every and (it % log_every == 0 or it == steps - 1):
            s = sums.cpu().numpy()
            hist.append((it, float(s[0] / max(s[1], 1.0))))
    net.check()
    return hist


def predict(net, q_dev, chunk=None):
    """Predicted distances as a (N, 24) device tensor (compare them after clip())."""
    import torch
    N = q_dev.shape[0]
    chunk = chunk or net.cap
    out = torch.empty((N, 24), dtype=torch.float32, device="cuda")
    for s in range(0, N, chunk):
        net.forward(q_dev[s:s + chunk].contiguous(), out[s:s + chunk])
    net.check()
    return out


def cached_labels(lab, q, path):
    """lab(q), kept in an .npz file: read back when the file holds labels of exactly these
    joint states (a SHA-1 of q is stored with them), else computed and written."""
    import hashlib
    q = np.ascontiguousarray(q, dtype=np.float64)
    key = hashlib.sha1(q.tobytes()).hexdigest()
    if os.path.exists(path):
        with np.load(path) as z:
            if str(z["key"]) == key:
                return z["dist"], z["status"]
    d, s = lab(q)
    np.savez(path, key=np.array(key), dist=d, status=s)
    return d, s


def near_weights(y, near_weight=3.0, scale=0.05):
    """Per-entry loss weights: 1 + near_weight exp(-y / scale), so errors on distances
    that decide a fallback (a few cm) count up to 1 + near_weight times more.  The
    kernels' masked loss takes the weight as its mask: the gradient is that of the
    weighted mean squared error."""
    return 1.0 + near_weight * np.exp(-np.asarray(y) / scale)


def fit(lab, net, n_train, n_val, seed, steps, batch=8192, lr=2e-3, near_weight=3.0, log_every=0):
    """Labels n_train + n_val seeded configurations on the exact path, trains `net` on
    the clipped valid distances (weighted toward small distances, `near_weights`) and
    returns (history, validation EvalResult, the safety margin = 5 cm + validation max
    error, label throughput in configurations/s, the per-sphere margins of
    `sphere_margins` on the validation set)."""
    import torch
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    q_tr = synth.joint_states(seed, n_train)
    t0 = time.perf_counter()
    d_tr, s_tr = lab(q_tr)
    label_qps = n_train / (time.perf_counter() - t0)
    m_tr = lab.valid_mask(s_tr)
    y_tr = np.where(m_tr, clip(d_tr), 0)
    w_tr = np.where(m_tr, near_weights(y_tr, near_weight), 0.0)
    hist = train(net, dev(q_tr), dev(y_tr), dev(w_tr), steps=steps, batch=batch, lr=lr, log_every=log_every)
    q_va = synth.joint_states(seed + 1, n_val)
    d_va, s_va = lab(q_va)
    p_va, y_va, m_va = clip(predict(net, dev(q_va)).cpu().numpy()), clip(d_va), lab.valid_mask(s_va)
    r_va = evaluate(p_va, y_va, m_va)
    return hist, r_va, 0.05 + r_va.max_err_mm / 1000.0, label_qps, sphere_margins(p_va, y_va, m_va)


def throughput(fn, n_items, reps=5, warmup=2):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        fn()
    torch.cuda.synchronize()
    return n_items * reps / (time.perf_counter() - t0)


def _main():
    """`python -m paper_2407_02363_b300.surrogate forward [--batch B] [--reps R]`: runs the
    surrogate forward on seeded random joint angles (He-uniform weights), for timing and
    profiling; prints ms per batch."""
    import argparse

    import torch

    from . import build
    ap = argparse.ArgumentParser()
    ap.add_argument("mode", choices=("forward",))
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--reps", type=int, default=10)
    a = ap.parse_args()
    build.build()
    rng = np.random.default_rng(0)
    net = v.MLP(a.batch)
    params = []
    for i, o in zip((14, 256, 256, 256, 256), (256, 256, 256, 256, 24)):
        params += [rng.uniform(-math.sqrt(6 / i), math.sqrt(6 / i), o * i), np.zeros(o)]
    net.set_params(np.concatenate(params).astype(np.float32))
    q = torch.from_numpy(synth.joint_states(1, a.batch).astype(np.float32)).cuda()
    out = torch.empty((a.batch, 24), device="cuda")
    for _ in range(3):
        net.forward(q, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        net.forward(q, out)
    e1.record()
    torch.cuda.synchronize()
    net.check()
    print(f"forward batch {a.batch}: {e0.elapsed_time(e1) / a.reps:.4f} ms")
    net.close()


if __name__ == "__main__":
    _main()
