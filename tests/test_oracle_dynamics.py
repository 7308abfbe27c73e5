"""Pins of the oracle's unicycle layer: SI -> unicycle map, wheel clip, Euler integration.

The unicycle model (paper Sec. 4.1) under constant (v, omega) with explicit Euler has a closed
form: theta_k = theta_0 + k omega dt and
    (x_k + i y_k) = (x_0 + i y_0) + v dt e^{i theta_0} (1 - e^{i k omega dt}) / (1 - e^{i omega dt}).
The SI -> unicycle map is pinned by the kinematic fact it is built on: the point l ahead of the
axle moves with the commanded SI velocity.
"""
import numpy as np
import pytest

import oracle

C = oracle.default_cfg()


def _u_for(v, w, th, l=0.05):
    """SI velocity whose unicycle image is (v, w): the inverse of the 2x2 map."""
    return v * np.cos(th) - l * w * np.sin(th), v * np.sin(th) + l * w * np.cos(th)


@pytest.mark.parametrize("v,w,th0", [(0.15, 0.8, 0.4), (0.08, -2.0, -2.9), (0.02, 3.0, 3.1),
                                     (0.18, 0.0, 1.0), (-0.12, 0.7, -0.3)])
def test_euler_arc_closed_form(v, w, th0):
    # |v| + |w| L/2 <= vmax: inside the wheel limits, so the clip leaves (v, w) unchanged
    pose = np.array([0.3, -0.2, th0])
    x0, y0 = pose[0], pose[1]
    dt = C["dt"]
    K = 60
    for k in range(1, K + 1):
        ux, uy = _u_for(v, w, pose[2])
        pose, vw = oracle.unicycle_update(C, ux, uy, pose)
        assert abs(vw[0] - v) < 1e-12 and abs(vw[1] - w) < 1e-12
        if w != 0.0:
            z = (x0 + 1j * y0) + v * dt * np.exp(1j * th0) * (1 - np.exp(1j * k * w * dt)) / (
                1 - np.exp(1j * w * dt))
        else:
            z = (x0 + 1j * y0) + k * v * dt * np.exp(1j * th0)
        assert abs(pose[0] - z.real) < 1e-12 and abs(pose[1] - z.imag) < 1e-12
        dth = (pose[2] - (th0 + k * w * dt) + np.pi) % (2 * np.pi) - np.pi
        assert abs(dth) < 1e-12
        assert -np.pi <= pose[2] <= np.pi


def test_euler_converges_to_continuous_circle():
    v, w = 0.1, 1.0
    errs = []
    for dt in (0.01, 0.005, 0.0025):
        c = dict(C, dt=dt)
        pose = np.array([0.0, 0.0, 0.0])
        steps = int(round(1.0 / dt))
        for _ in range(steps):
            pose, _ = oracle.unicycle_update(c, *_u_for(v, w, pose[2]), pose)
        # exact: circle of radius v/w
        xe, ye = (v / w) * np.sin(w * 1.0), (v / w) * (1 - np.cos(w * 1.0))
        errs.append(np.hypot(pose[0] - xe, pose[1] - ye))
    assert errs[0] / errs[1] > 1.8 and errs[1] / errs[2] > 1.8  # first order


@pytest.mark.parametrize("th", [0.0, 0.7, -2.2, 3.0])
def test_projected_point_moves_with_si_velocity(th):
    c = dict(C, dt=1e-7, wmax=1e6, vmax=10.0)
    ux, uy = 0.13, -0.08
    pose = np.array([0.2, 0.1, th])
    p0 = pose[:2] + 0.05 * np.array([np.cos(th), np.sin(th)])
    p1pose, _ = oracle.unicycle_update(c, ux, uy, pose)
    p1 = p1pose[:2] + 0.05 * np.array([np.cos(p1pose[2]), np.sin(p1pose[2])])
    vel = (p1 - p0) / 1e-7
    assert np.allclose(vel, [ux, uy], atol=1e-5)


@pytest.mark.parametrize("v,w,ve,we", [
    (0.3, 0.0, 0.2, 0.0),      # both wheels at +vmax
    (0.0, 5.0, 0.0, 3.6),      # pure rotation limited to wmax
    (0.2, 3.6, 0.1, 1.8),      # right wheel saturates at vmax, left at 0
    (0.1, 1.0, 0.1, 1.0),      # inside the limits: unchanged
    (-0.25, -1.0, None, None),  # one wheel saturates in reverse
])
def test_wheel_clip_special_cases(v, w, ve, we):
    L = 2 * 0.2 / 3.6
    pose = np.array([0.0, 0.0, 0.0])
    _, vw = oracle.unicycle_update(C, v, 0.05 * w, pose)
    if we is None:
        # (-0.25, -1): wr = -0.25 - L/2 -> -0.2, wl = -0.25 + L/2 = -0.1944 -> kept
        wr, wl = -0.2, -0.25 + 0.5 * L
        ve, we = 0.5 * (wr + wl), (wr - wl) / L
    assert abs(vw[0] - ve) < 1e-12 and abs(vw[1] - we) < 1e-12
