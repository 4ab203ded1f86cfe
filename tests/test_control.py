"""The task-priority collision-avoidance controller (Sec. III-F) on the CPU: the position
Jacobian against finite differences of forward kinematics, the activation function's
cases, the regularised task-priority solution's defining properties, and a closed loop
with analytic nearest obstacle points in which the controller keeps every bounding
sphere clear of a sweeping obstacle that hits the arm without it."""
import numpy as np

import oracle
from paper_2407_02363_b300 import control as C
from paper_2407_02363_b300 import synth


def test_position_jacobian_matches_finite_differences():
    chain = synth.make_chain(5, (0.5, 0.5, 0.2))
    rng = np.random.default_rng(0)
    for _ in range(5):
        q = rng.uniform(-np.pi, np.pi, chain.n_joints)
        P = oracle.fk(chain, q)
        link = int(rng.integers(1, chain.n_joints + 1))
        local = rng.normal(0, 0.1, 3)
        p = P[link][:, :3] @ local + P[link][:, 3]
        J = C.position_jacobian(P, link, p)
        h = 1e-6
        for j in range(chain.n_joints):
            dq = np.zeros(chain.n_joints)
            dq[j] = h
            Pp, Pm = oracle.fk(chain, q + dq), oracle.fk(chain, q - dq)
            num = ((Pp[link][:, :3] @ local + Pp[link][:, 3]) - (Pm[link][:, :3] @ local + Pm[link][:, 3])) / (2 * h)
            np.testing.assert_allclose(J[:, j], num, atol=1e-8)


def test_activation_cases_and_continuity():
    x_m, b = 0.1, 0.02
    assert C.activation(0.05, x_m, b) == 1.0 and C.activation(x_m, x_m, b) == 1.0
    assert C.activation(x_m + b, x_m, b) == 0.0 and C.activation(0.5, x_m, b) == 0.0
    assert abs(C.activation(x_m + b / 2, x_m, b) - 0.5) < 1e-12
    xs = np.linspace(0.09, 0.13, 4001)
    a = C.activation(xs, x_m, b)
    assert np.all(np.diff(a) <= 1e-12) and np.max(np.abs(np.diff(a))) < 2e-3


def test_task_priority_solution_properties():
    rng = np.random.default_rng(1)
    n = 7
    J = rng.normal(size=(3, n))
    xdot = rng.normal(size=3)
    qdot0 = rng.normal(size=n)
    # all tasks active, negligible regularisation: the tasks are met exactly and the
    # lower-priority motion only acts in their null space
    qd = C.task_priority(J, np.ones(3), xdot, qdot0, beta=1e-14, width=1e-9)
    np.testing.assert_allclose(J @ qd, xdot, atol=1e-9)
    pinv = np.linalg.pinv(J)
    np.testing.assert_allclose(qd - pinv @ xdot, (np.eye(n) - pinv @ J) @ qdot0, atol=1e-9)
    # no task active: the lower-priority motion passes unchanged
    np.testing.assert_allclose(C.task_priority(J, np.zeros(3), xdot, qdot0), qdot0, atol=1e-12)
    # near a singularity the regularisation keeps the joint velocity bounded
    Js = np.vstack([J[0], J[0] + 1e-4 * J[1]])
    big = C.task_priority(Js, np.ones(2), np.array([0.0, 1.0]), np.zeros(n), beta=1e-14, width=1e-9)
    reg = C.task_priority(Js, np.ones(2), np.array([0.0, 1.0]), np.zeros(n), beta=1e-2, width=1.0)
    assert np.linalg.norm(reg) < 1e-3 * np.linalg.norm(big)


def closed_loop_analytic(avoid, seed=3, n_frames=150, r_obs=0.12, dt=1 / 60):
    """The loop of control.run_closed_loop with the nearest obstacle point computed
    analytically (the obstacle is a sphere) instead of by the library."""
    p = C.AvoidanceParams()
    chain = synth.make_chain(seed, (0.96, 0.96, 0.25))
    sp = synth.sphere_model(chain)
    n = chain.n_joints
    q = np.array([0.4 * (-1) ** k for k in range(n)], float)
    tip_local = np.array([0.0, 0.0, chain.lengths[-1]])
    P0 = oracle.fk(chain, q)
    target = P0[n][:, :3] @ tip_local + P0[n][:, 3] + np.array([0.15, 0.1, -0.05])
    mid = P0[n // 2 + 1][:, 3]
    d = np.array([1.0, 0.3, 0.0]) / np.linalg.norm([1.0, 0.3, 0.0])
    m = len(sp.radius)
    worst = np.inf
    for f in range(n_frames):
        ctr = mid + (f / (n_frames - 1) - 0.5) * d
        P = oracle.fk(chain, q)
        R = P[sp.link]
        cen = np.einsum("nij,nj->ni", R[:, :, :3], sp.local) + R[:, :, 3]
        worst = min(worst, float((np.linalg.norm(cen - ctr, axis=1) - r_obs - sp.radius).min()))
        res = np.zeros(2 * m, dtype=[("status", "i4"), ("nearest", "f4", (3,))])
        for i in range(m):
            v = cen[i] - ctr
            res[i]["nearest"] = ctr + r_obs * v / np.linalg.norm(v)
        res[m:]["status"] = 2          # no self obstacle in this test
        qd0, _ = C.reach_velocity(P, n, tip_local, target)
        if avoid:
            J, A, ref = C.avoidance_tasks(res, cen, sp.radius, P, sp, p)
            qd = C.task_priority(J, A, ref, qd0, p.beta, p.width)
        else:
            qd = qd0
        q = q + dt * np.clip(qd, -2.0, 2.0)
    return worst


def test_closed_loop_keeps_clearance_that_is_lost_without_avoidance():
    for seed in (3, 5, 7):
        assert closed_loop_analytic(True, seed) > 0.02
        assert closed_loop_analytic(False, seed) < -0.05
