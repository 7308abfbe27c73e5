"""Pins of the oracle's unicycle pose controller (the paper's Sec. 4.2 evaluates a pose
controller without giving its law, so the published posture-regulation law of Aicardi et al.
(1995) stands for it) and of its plumbing into the Navigation step (CPU only).

The law's defining property is the Lyapunov function V = (rho^2 + gam^2 + k3 del^2) / 2 of the
polar coordinates (distance to the goal, angle from the heading to the goal direction, angle of
that direction in the goal's frame) with dV/dt = -k1 cos^2(gam) rho^2 - k2 gam^2 along the
unicycle's motion.  The tests measure V geometrically from poses and integrate the unicycle
kinematics themselves, so a sign, frame or term error in the law shows as a wrong rate.
"""
import numpy as np
import pytest

import oracle


def _wrap(a):
    return (a + np.pi) % (2 * np.pi) - np.pi


def _polar(pose, goal, k3):
    """rho, gam, del and V from the geometry (the goal's frame built here, independently)."""
    c, s = np.cos(goal[2]), np.sin(goal[2])
    dx, dy = pose[0] - goal[0], pose[1] - goal[1]
    xr, yr = c * dx + s * dy, -s * dx + c * dy
    thr = _wrap(pose[2] - goal[2])
    rho = np.hypot(xr, yr)
    to_goal = np.arctan2(-yr, -xr)          # direction from the robot to the goal, goal frame
    gam = _wrap(to_goal - thr)
    dl = _wrap(to_goal)
    return rho, gam, dl, 0.5 * (rho ** 2 + gam ** 2 + k3 * dl ** 2)


def _advance(pose, v, w, dt):
    """Exact unicycle motion under constant (v, w) for dt (arc)."""
    x, y, th = pose
    if abs(w) < 1e-12:
        return np.array([x + v * dt * np.cos(th), y + v * dt * np.sin(th), th])
    return np.array([x + v / w * (np.sin(th + w * dt) - np.sin(th)),
                     y - v / w * (np.cos(th + w * dt) - np.cos(th)), th + w * dt])


@pytest.mark.parametrize("gains", [(1.0, 2.0, 1.0), (0.5, 3.0, 2.0)])
def test_lyapunov_rate_matches_closed_form(gains):
    k1, k2, k3 = gains
    c = oracle.default_cfg(pose_k1=k1, pose_k2=k2, pose_k3=k3)
    rng = np.random.default_rng(3)
    checked = 0
    for _ in range(400):
        pose = np.array([*rng.uniform(-1.5, 1.5, 2), rng.uniform(-np.pi, np.pi)])
        goal = np.array([*rng.uniform(-1.5, 1.5, 2), rng.uniform(-np.pi, np.pi)])
        rho, gam, dl, V0 = _polar(pose, goal, k3)
        if rho < 0.05 or abs(abs(gam) - np.pi) < 0.05 or abs(abs(dl) - np.pi) < 0.05:
            continue  # away from the polar singularity and the angle wrap
        v, w = oracle.pose_control(c, pose, goal)
        h = 1e-6
        _, _, _, V1 = _polar(_advance(pose, v, w, h), goal, k3)
        rate = (V1 - V0) / h
        expect = -k1 * np.cos(gam) ** 2 * rho ** 2 - k2 * gam ** 2
        assert abs(rate - expect) < 1e-4 * (1 + abs(expect)), (pose, goal, rate, expect)
        assert rate <= 1e-6
        checked += 1
    assert checked > 300


def test_special_cases_and_frame_invariance():
    c = oracle.default_cfg(pose_k1=1.0, pose_k2=2.0, pose_k3=1.0)
    # heading straight at the goal point (gam = 0): v = k1 rho, omega = k1 k3 del
    goal = np.array([0.0, 0.0, 0.3])
    pose = np.array([-1.0, 0.0, 0.0])          # goal dead ahead, 1 m away
    v, w = oracle.pose_control(c, pose, goal)
    assert abs(v - 1.0) < 1e-15
    assert abs(w - (0.0 - 0.3) * 1.0) < 1e-12   # del = direction (0) minus goal heading (0.3)
    # on the goal point: no translation, turn towards the goal heading
    v, w = oracle.pose_control(c, np.array([0.0, 0.0, 1.0]), goal)
    assert v == 0.0 and abs(w - (-2.0 * 0.7)) < 1e-12
    # rotating and translating the world leaves the command unchanged
    rng = np.random.default_rng(8)
    for _ in range(50):
        pose = np.array([*rng.uniform(-1, 1, 2), rng.uniform(-np.pi, np.pi)])
        goal = np.array([*rng.uniform(-1, 1, 2), rng.uniform(-np.pi, np.pi)])
        a, t = rng.uniform(-np.pi, np.pi), rng.uniform(-2, 2, 2)
        R = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
        p2 = np.array([*(R @ pose[:2] + t), pose[2] + a])
        g2 = np.array([*(R @ goal[:2] + t), goal[2] + a])
        assert np.allclose(oracle.pose_control(c, pose, goal), oracle.pose_control(c, p2, g2),
                           atol=1e-9)


def test_closed_loop_reaches_the_goal_pose():
    c = oracle.default_cfg(pose_k1=1.0, pose_k2=2.0, pose_k3=1.0)
    rng = np.random.default_rng(11)
    for _ in range(20):
        pose = np.array([*rng.uniform(-1.2, 1.2, 2), rng.uniform(-np.pi, np.pi)])
        goal = np.array([*rng.uniform(-1.2, 1.2, 2), rng.uniform(-np.pi, np.pi)])
        for _ in range(6000):
            v, w = oracle.pose_control(c, pose, goal)
            pose = _advance(pose, v, w, 0.005)
        assert np.hypot(*(pose[:2] - goal[:2])) < 1e-3
        assert abs(_wrap(pose[2] - goal[2])) < 1e-2


def test_navigation_step_uses_the_pose_law():
    """controller = pose: u_nom is the SI velocity of the projected point under the law's
    (v, omega), capped, plus the noise, capped; goal headings come from the goal draw."""
    N, E, seed = 4, 32, 5
    c = oracle.default_cfg(n_max=N, controller=1, noise_amp=0.0)
    s = oracle.reset(c, seed, [N] * E)
    f32 = np.float32
    for e in range(3):
        for i in range(N):
            w = oracle.philox4x32_10([e, 0, (3 << 24) | i, 0], [seed, 0])
            u = f32(np.uint32(w[2]) >> np.uint32(8)) * f32(2.0 ** -24)
            assert s.gth[N * e + i] == float(-f32(np.pi) + u * f32(2 * np.pi))
    for _ in range(3):
        oracle.step(c, seed, s)
    before = s.copy()
    _, _, _, tr = oracle.step(c, seed, s, trace=True)
    for g in range(N * E):
        th = before.th[g]
        v, w = oracle.pose_control(c, [before.x[g], before.y[g], th],
                                   [before.gx[g], before.gy[g], before.gth[g]])
        u = np.array([v * np.cos(th) - 0.05 * w * np.sin(th), v * np.sin(th) + 0.05 * w * np.cos(th)])
        n = np.hypot(*u)
        if n > 0.2:
            u *= 0.2 / n
        assert np.allclose(tr["u_nom"][g], u, atol=1e-15, rtol=0)
    # the SI velocity maps back to the law's (v, omega) when no cap applies
    cw = oracle.default_cfg(n_max=N, controller=1, noise_amp=0.0, vmax=1e3, wmax=1e6)
    s = oracle.reset(cw, seed, [N] * E)
    before = s.copy()
    _, _, _, tr = oracle.step(cw, seed, s, trace=True)
    for g in range(8):
        th = before.th[g]
        v, w = oracle.pose_control(cw, [before.x[g], before.y[g], th],
                                   [before.gx[g], before.gy[g], before.gth[g]])
        ux, uy = tr["u_nom"][g]
        assert abs(np.cos(th) * ux + np.sin(th) * uy - v) < 1e-12
        assert abs((-np.sin(th) * ux + np.cos(th) * uy) / 0.05 - w) < 1e-9


def test_pose_controller_rejected_outside_navigation():
    with pytest.raises(Exception):
        oracle.reset(oracle.default_cfg(oracle.FORAGE, n_max=4, controller=1), 1, [4] * 4)
    with pytest.raises(Exception):
        oracle.reset(oracle.default_cfg(n_max=4, controller=1, pose_k2=0.0), 1, [4] * 4)
