"""Task-priority collision-avoidance controller (Sec. III-D to III-F, Algs. 2-3): the CPU
consumer of the distance queries.  Per control cycle, for every bounding sphere i with
centre C_i and nearest obstacle voxel O_i (from the environment map, and O_si from the
self map):
  * x_i = ||O_i - C_i||, the scalar avoidance task (Eq. (dist));
  * J_i = -((O_i - C_i) / x_i)^T J_ci(q), J_ci the position Jacobian at C_i (Eq. (jac));
  * reference rate kappa (x* - x_i) (Eq. (ref_vel));
  * activation A_ii: 1 while the sphere is inside its threshold, the cosine transition of
    the paper over a buffer b, 0 beyond;
  * joint velocity from the regularised task-priority solution (Eq.
    (task_oriented_solution)), with a lower-priority joint velocity qdot0 (here a
    reaching task for the last link) in the null space of the active avoidance tasks.

Plain numpy; the distances come from the CUDA library through vedt.Map.frame_host.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def joint_axes(poses):
    """World origin o_k and rotation axis z_k of joints k = 1..n from link poses
    (n+1, 3, 4): joint k turns link k about its frame's z axis, which Rz(q_k) leaves in
    place, so both are read from the pose of link k."""
    P = np.asarray(poses, dtype=np.float64)
    return P[1:, :, 3].copy(), P[1:, :, 2].copy()


def position_jacobian(poses, link, p):
    """3 x n position Jacobian of the world point p fixed to link `link` (1..n):
    column j is z_j x (p - o_j) for revolute joints j <= link, zero beyond."""
    o, z = joint_axes(poses)
    n = o.shape[0]
    J = np.zeros((3, n))
    for j in range(min(int(link), n)):
        J[:, j] = np.cross(z[j], np.asarray(p, np.float64) - o[j])
    return J


def activation(x, x_m, b):
    """A_ii for an inequality task x >= x_m with transition buffer b > 0: 1 at or inside
    the threshold, (1 + cos(pi (x - x_m) / b)) / 2 across the buffer, 0 beyond it."""
    x = np.asarray(x, np.float64)
    a = 0.5 * (np.cos(np.pi * (x - x_m) / b) + 1.0)
    return np.where(x <= x_m, 1.0, np.where(x >= x_m + b, 0.0, a))


def bell(sigma, beta, width):
    """Regularisation weight of a singular value: largest (beta) at 0, decaying with a
    Gaussian bell of the given width."""
    return beta * np.exp(-(np.asarray(sigma, np.float64) / width) ** 2)


def task_priority(J, A, xdot_ref, qdot0, beta=1e-3, width=1e-2):
    """qdot = G J^T A A xdot + (I - G J^T A A J) qdot0, G = (J^T A J + V P V^T)^#, with
    J^T A J = U S V^T and P = bell(singular values of J), zero where J has none: the
    minimiser of ||A (xdot - J qdot)||^2 + ||J qdot||^2_{A (I - A)} + ||V^T qdot||^2_P plus
    the null-space motion."""
    J = np.atleast_2d(np.asarray(J, np.float64))
    n = J.shape[1]
    if J.shape[0] == 0:
        return np.asarray(qdot0, np.float64).copy()
    A = np.diag(np.asarray(A, np.float64)) if np.ndim(A) == 1 else np.asarray(A, np.float64)
    M = J.T @ A @ J
    _, S, Vt = np.linalg.svd(M)
    # the singular values of A^(1/2) J are sqrt(S); directions past the task count have no
    # singular value of J and take no regularisation
    p = bell(np.sqrt(np.maximum(S, 0.0)), beta, width)
    p[min(J.shape[0], n):] = 0.0
    R = Vt.T @ np.diag(p) @ Vt
    G = np.linalg.pinv(M + R)
    W = J.T @ A @ A
    return G @ W @ np.asarray(xdot_ref, np.float64) + (np.eye(n) - G @ W @ J) @ np.asarray(qdot0, np.float64)


def reach_velocity(poses, link, p_local, target, gain=2.0, damping=1e-2):
    """Damped least-squares joint velocity moving a point of `link` towards `target`."""
    T = np.asarray(poses, np.float64)[link]
    p = T[:, :3] @ np.asarray(p_local, np.float64) + T[:, 3]
    J = position_jacobian(poses, link, p)
    e = gain * (np.asarray(target, np.float64) - p)
    return J.T @ np.linalg.solve(J @ J.T + damping ** 2 * np.eye(3), e), p


@dataclass
class AvoidanceParams:
    margin: float = 0.08     # activation threshold x_M = sphere radius + margin
    buffer: float = 0.02     # b (the paper's 2 cm for collision avoidance); x* = x_M + b
    kappa: float = 8.0       # reference-rate gain
    beta: float = 1e-3
    width: float = 1e-2


def avoidance_tasks(results, centres, radii, poses, spheres, params, self_mask=None):
    """Rows of the active avoidance tasks from one cycle's sphere results (vedt
    SPHERE_DTYPE: env block then self block of m each): Jacobian rows, activations and
    reference rates.  Spheres with no obstacle, outside the grid, or masked for the self
    map contribute no row."""
    m = len(radii)
    P = np.asarray(poses, np.float64)
    n = P.shape[0] - 1
    o, z = joint_axes(P)
    C = np.asarray(centres, np.float64)
    links = np.asarray(spheres.link, np.int64)
    # position Jacobians of all sphere centres: (m, 3, n), column j zero past the link
    Jc = np.cross(z[None, :, :], C[:, None, :] - o[None, :, :])          # (m, n, 3)
    Jc = np.where((np.arange(n)[None, :] < links[:, None])[:, :, None], Jc, 0.0).transpose(0, 2, 1)
    res = np.asarray(results)
    keep = np.ones(2 * m, bool)
    if self_mask is not None:
        keep[m:] = np.asarray(self_mask, bool)
    keep &= res["status"] == 0
    O = res["nearest"].astype(np.float64)
    sph = np.concatenate([np.arange(m), np.arange(m)])
    d = O - C[sph]
    x = np.linalg.norm(d, axis=1)
    x_m = np.asarray(radii, np.float64)[sph] + params.margin
    a = activation(x, x_m, params.buffer)
    keep &= (a > 0.0) & (x > 0.0)
    idx = np.nonzero(keep)[0]
    u = d[idx] / x[idx, None]
    rows = -np.einsum("ka,kaj->kj", u, Jc[sph[idx]])
    return rows.reshape(-1, n), a[idx], params.kappa * (x_m[idx] + params.buffer - x[idx])


def fibonacci_sphere(n, radius):
    """n points spread evenly over a sphere surface (golden-angle spiral)."""
    k = np.arange(n) + 0.5
    z = 1.0 - 2.0 * k / n
    r = np.sqrt(1.0 - z * z)
    phi = np.pi * (3.0 - np.sqrt(5.0)) * k
    return radius * np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def run_closed_loop(v, n_frames=150, avoid=True, seed=3, dims=(96, 96, 96), vs=0.02, dt=1.0 / 60.0,
                    obstacle_radius=0.12, params=None, sphere_rule="fixed"):
    """A synthetic closed loop (Alg. 2 with Alg. 3 as the consumer): a 7-DoF arm reaches
    for a target while a spherical obstacle (its surface as a point cloud) sweeps through
    the arm.  Every cycle runs one library frame (clear, insert links and cloud, EDT of
    both maps, sphere queries) and one controller step.  Returns the smallest geometric
    clearance between any bounding sphere and the obstacle over the run, and the final
    distance of the reaching point to its target.  sphere_rule: "fixed" (24 spheres of
    5 cm spread by link length) or "obb" (the OBB sphere rows of Sec. III-B)."""
    from . import synth
    params = params or AvoidanceParams()
    grid = synth.GridSpec(tuple(dims), vs)
    ext = np.array(grid.extent)
    chain = synth.make_chain(seed, (ext[0] / 2, ext[1] / 2, 0.25))
    models = synth.link_models(chain, vs)
    if sphere_rule == "obb":
        from .spheres import sphere_model_obb
        spheres = sphere_model_obb(models)
    elif sphere_rule == "fixed":
        spheres = synth.sphere_model(chain)
    else:
        raise ValueError(f"unknown sphere rule {sphere_rule!r}")
    n = chain.n_joints
    m = v.Map(grid.dims, grid.voxel_size, grid.origin)
    m.register_links(models)
    cchain = v.make_chain(chain)
    self_mask = ~np.asarray(spheres.acm, bool)
    q = np.array([0.4 * (-1) ** k for k in range(n)], np.float64)
    tip_local = np.array([0.0, 0.0, float(chain.lengths[-1])])
    P0 = v.fk(chain, q)
    tip0 = P0[n][:, :3] @ tip_local + P0[n][:, 3]
    target = tip0 + np.array([0.15, 0.1, -0.05])
    mid = P0[n // 2 + 1][:, 3]
    surf = fibonacci_sphere(2000, obstacle_radius)
    direction = np.array([1.0, 0.3, 0.0]) / np.linalg.norm([1.0, 0.3, 0.0])
    min_clear = np.inf
    tip = tip0
    for f in range(n_frames):
        ctr = mid + (f / max(n_frames - 1, 1) - 0.5) * 1.0 * direction
        cloud = (surf + ctr).astype(np.float32)
        poses = v.fk(chain, q)
        centres = v.sphere_centres(cchain, spheres, q)
        res = m.frame_host(cloud, cchain, q, 0b111, centres, spheres.radius)
        gap = np.linalg.norm(centres.astype(np.float64) - ctr, axis=1) - obstacle_radius - spheres.radius
        min_clear = min(min_clear, float(gap.min()))
        qdot0, tip = reach_velocity(poses, n, tip_local, target)
        if avoid:
            J, A, ref = avoidance_tasks(res, centres, spheres.radius, poses, spheres, params, self_mask)
            qdot = task_priority(J, A, ref, qdot0, params.beta, params.width)
        else:
            qdot = qdot0
        qdot = np.clip(qdot, -2.0, 2.0)
        q = q + dt * qdot
    m.close()
    return {"min_clearance_m": min_clear, "tip_error_m": float(np.linalg.norm(target - tip)), "frames": n_frames,
            "spheres": int(len(spheres.radius))}
