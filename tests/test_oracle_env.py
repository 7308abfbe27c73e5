"""Pins of the oracle's environment layer: nominal control, flags, rewards, observations,
episodes and auto-reset, foraging rule, forward invariance of the barrier (CPU only).

Scenario definitions follow paper App. B (Navigation: position, goal, distance reward;
Foraging: robots within the radius whose summed level reaches the resource level forage it,
reward = the resource's level; max steps 100).
"""
import itertools

import numpy as np
import pytest

import oracle


def _proj(s, l=0.05):
    return s.x + l * np.cos(s.th), s.y + l * np.sin(s.th)


def _wrap(a):
    return (a + np.pi) % (2 * np.pi) - np.pi


def _ang_close(a, b, tol):
    return np.all(np.abs(_wrap(np.asarray(a) - np.asarray(b))) < tol)


def test_navigation_reward_flags_and_obs_recomputed():
    N, E = 4, 64
    c = oracle.default_cfg(n_max=N, episode_len=10_000)
    s = oracle.reset(c, 9, [N] * E)
    for _ in range(25):
        oracle.step(c, 9, s)
    before = s.copy()
    obs, rew, done, tr = oracle.step(c, 9, s, trace=True)
    assert not done.any()
    p0x, p0y = _proj(before)
    p1x, p1y = _proj(s)
    for e in range(E):
        sl = slice(4 * e, 4 * e + 4)
        d0 = np.hypot(p0x[sl] - before.gx[sl], p0y[sl] - before.gy[sl])
        d1 = np.hypot(p1x[sl] - s.gx[sl], p1y[sl] - s.gy[sl])
        col = sum(1 for i, j in itertools.combinations(range(N), 2)
                  if (p1x[sl][i] - p1x[sl][j]) ** 2 + (p1y[sl][i] - p1y[sl][j]) ** 2 < 0.17 ** 2)
        assert abs(rew[e] - (-(d1 - d0).sum() - 1.0 * col)) < 1e-12
        for i in range(N):
            o = obs[4 * e + i]
            g = 4 * e + i
            assert np.array_equal(o[:5], [s.x[g], s.y[g], s.th[g], s.gx[g], s.gy[g]])
            others = [j for j in range(N) if j != i]
            for slot, j in enumerate(others):
                gj = 4 * e + j
                rel = o[5 + 3 * slot:8 + 3 * slot]
                assert abs(rel[0] - (s.x[gj] - s.x[g])) < 1e-15
                assert abs(rel[1] - (s.y[gj] - s.y[g])) < 1e-15
                assert _ang_close(rel[2], s.th[gj] - s.th[g], 1e-12) and abs(rel[2]) <= np.pi
    # antisymmetry of the relative blocks: robot i sees j at -(what j sees of i)
    o = obs.reshape(E, N, -1)
    assert np.allclose(o[:, 0, 5:7], -o[:, 1, 5:7], atol=1e-15)


def test_scripted_nominal_control_recomputed_from_generator():
    N, E, seed = 4, 16, 0xBEEF
    c = oracle.default_cfg(n_max=N)
    s = oracle.reset(c, seed, [N] * E)
    for _ in range(3):
        oracle.step(c, seed, s)
    before = s.copy()
    _, _, _, tr = oracle.step(c, seed, s, trace=True)
    px, py = _proj(before)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    f32 = np.float32
    for e in range(E):
        for i in range(N):
            g = N * e + i
            ux, uy = before.gx[g] - px[g], before.gy[g] - py[g]
            nrm = np.hypot(ux, uy)
            if nrm > 0.2:
                ux, uy = ux * 0.2 / nrm, uy * 0.2 / nrm
            w = oracle.philox4x32_10([e, before.ep[e], (1 << 24) | (i >> 1), before.t[e]], key)
            u = [f32(np.uint32(v) >> np.uint32(8)) * f32(2.0 ** -24) for v in w]
            ex = (u[2 * (i & 1)] - f32(0.5)) * f32(0.1)
            ey = (u[2 * (i & 1) + 1] - f32(0.5)) * f32(0.1)
            ux, uy = ux + float(ex), uy + float(ey)
            nrm = np.hypot(ux, uy)
            if nrm > 0.2:
                ux, uy = ux * 0.2 / nrm, uy * 0.2 / nrm
            assert np.allclose(tr["u_nom"][g], [ux, uy], atol=1e-15, rtol=0)


def test_noise_statistics():
    # far from goals the capped direction plus U(-0.05, 0.05)^2 noise: the noise sample mean is 0
    N, E = 4, 512
    c = oracle.default_cfg(n_max=N, k_si=0.0)  # nominal = noise only
    s = oracle.reset(c, 2, [N] * E)
    _, _, _, tr = oracle.step(c, 2, s, trace=True)
    u = tr["u_nom"]
    assert np.all(np.abs(u) <= 0.05) and abs(u.mean()) < 0.004
    assert abs(u.std() - 0.1 / np.sqrt(12)) < 0.003


def test_episode_done_and_auto_reset():
    N, E, T = 4, 8, 5
    c = oracle.default_cfg(n_max=N, episode_len=T)
    s = oracle.reset(c, 4, [N] * E)
    for t in range(T - 1):
        _, _, done, _ = oracle.step(c, 4, s)
        assert not done.any()
    obs, _, done, _ = oracle.step(c, 4, s)
    assert done.all()
    fresh = oracle.reset(c, 4, [N] * E, ep=[1] * E)
    assert np.array_equal(s.x, fresh.x) and np.array_equal(s.th, fresh.th)
    assert np.all(s.t == 0) and np.all(s.ep == 1)
    assert np.all(s.counters.reshape(E, 8)[:, oracle.CNT_EPISODES] == 1)
    assert np.array_equal(obs[:, 0], fresh.x)  # obs after done describe the new episode


def test_rollout_equals_repeated_steps_and_is_deterministic():
    N, E, T = 4, 8, 130
    c = oracle.default_cfg(n_max=N)
    a = oracle.reset(c, 8, [N] * E)
    b = a.copy()
    obs_r, rew_r, done_r = oracle.rollout(c, 8, a, T)
    for t in range(T):
        obs, rew, done, _ = oracle.step(c, 8, b)
        assert np.array_equal(obs, obs_r[t]) and np.array_equal(rew, rew_r[t])
        assert np.array_equal(done, done_r[t])
    assert np.array_equal(a.x, b.x) and np.array_equal(a.counters, b.counters)
    assert done_r.sum(0).tolist() == [1] * E


@pytest.mark.parametrize("N,E,kw", [(4, 256, {}), (10, 64, {}),
                                    (20, 32, dict(near_frac=0.3, wmax=1e4))])
def test_forward_invariance_from_safe_starts(N, E, kw):
    """From a safe start the barrier keeps every pair of projected points at least r apart.
    For N = 20 the wheel clip (which acts after the QP) is disabled: with the clip the
    continuous-time guarantee does not carry over to dense crowds."""
    c = oracle.default_cfg(n_max=N, **kw)
    s = oracle.reset(c, 13, [N] * E)
    mind = np.inf
    for _ in range(150):
        oracle.step(c, 13, s)
        px, py = _proj(s)
        P, Q = px.reshape(E, N), py.reshape(E, N)
        d = np.hypot(P[:, :, None] - P[:, None], Q[:, :, None] - Q[:, None]) + 9 * np.eye(N)
        mind = min(mind, d.min())
    cnt = s.counters.reshape(E, 8)
    assert cnt[:, oracle.CNT_QP_ACTIVE].sum() > 0
    assert cnt[:, oracle.CNT_QP_INFEASIBLE].sum() == 0
    assert mind >= 0.17 - 2e-3
    assert cnt[:, oracle.CNT_COLLISIONS].sum() == 0


def _forage_by_subsets(levels, inside, qlevel):
    """Paper App. B: foraged iff some set of robots inside the radius has summed level >= the
    resource level.  Enumerate every subset."""
    idx = [i for i in range(len(levels)) if inside[i]]
    for k in range(1, len(idx) + 1):
        for S in itertools.combinations(idx, k):
            if sum(levels[i] for i in S) >= qlevel:
                return True
    return False


def test_foraging_rule_by_subset_enumeration():
    c = oracle.default_cfg(oracle.FORAGE, n_max=6, episode_len=10_000, forage_radius=0.6)
    n = np.array([2, 3, 4, 5, 6] * 12, np.int32)
    E = len(n)
    s = oracle.reset(c, 17, n)
    seen = 0
    for _ in range(40):
        before = s.copy()
        _, rew, done, _ = oracle.step(c, 17, s)
        px, py = _proj(s)
        for e in range(E):
            if done[e]:
                continue
            sl = slice(int(s.off[e]), int(s.off[e + 1]))
            r_exp = 0.0
            for k in range(before.n_res[e]):
                g = e * 6 + k
                if not before.qactive[g]:
                    assert s.qactive[g] == 0
                    continue
                inside = (px[sl] - s.qx[g]) ** 2 + (py[sl] - s.qy[g]) ** 2 < 0.6 ** 2
                f = _forage_by_subsets(s.level[sl], inside, s.qlevel[g])
                assert bool(s.qactive[g] == 0) == f
                if f:
                    r_exp += s.qlevel[g]
                    seen += 1
            assert rew[e] == r_exp
    assert seen > 10


def test_foraging_done_when_all_foraged():
    c = oracle.default_cfg(oracle.FORAGE, n_max=3, episode_len=10_000, forage_radius=5.0)
    s = oracle.reset(c, 1, [3] * 16)
    _, rew, done, _ = oracle.step(c, 1, s)
    # radius covers the arena: every resource whose level <= summed robot levels goes at once
    assert done.sum() >= 1
    assert np.all(s.counters.reshape(16, 8)[:, oracle.CNT_SUCCESS] >= 2 * done)


def _goal_draw(seed, e, ep, i, ctr):
    """Goal of the reset's distribution under Philox counter word 3 = ctr (binary32 mapping)."""
    f32 = np.float32
    w = oracle.philox4x32_10([e, ep, (3 << 24) | i, ctr], [seed & 0xFFFFFFFF, seed >> 32])
    u = [f32(np.uint32(v) >> np.uint32(8)) * f32(2.0 ** -24) for v in w[:2]]
    lox, loy = f32(-1.6) + f32(0.2), f32(-1.0) + f32(0.2)
    wx, wy = (f32(1.6) - f32(0.2)) - lox, (f32(1.0) - f32(0.2)) - loy
    return float(lox + u[0] * wx), float(loy + u[1] * wy)


@pytest.mark.parametrize("eps", [0.05, 0.4])
def test_waypoint_goal_reassigned_on_arrival(eps):
    """Random Waypoint Navigation (Sec. 4.2): a robot whose new projected point lies strictly
    within goal_eps of its goal gets a new goal from the goal stream at counter t + 1; the others
    keep theirs; the reward of the step uses the old goals; each arrival is one success."""
    N, E, seed = 4, 24, 17
    c = oracle.default_cfg(n_max=N, episode_len=10_000, goal_eps=eps)
    s = oracle.reset(c, seed, [N] * E)
    # robot 0 of every env starts on its goal, so arrivals happen at once
    px, py = _proj(s)
    s.gx[0::N], s.gy[0::N] = px[0::N], py[0::N]
    arrivals = 0
    for _ in range(40):
        before = s.copy()
        _, rew, done, _ = oracle.step(c, seed, s)
        assert not done.any()
        p0x, p0y = _proj(before)
        p1x, p1y = _proj(s)
        for e in range(E):
            d_rew = 0.0
            for i in range(N):
                g = N * e + i
                d_rew -= (np.hypot(p1x[g] - before.gx[g], p1y[g] - before.gy[g])
                          - np.hypot(p0x[g] - before.gx[g], p0y[g] - before.gy[g]))
                d2 = (p1x[g] - before.gx[g]) ** 2 + (p1y[g] - before.gy[g]) ** 2
                assert abs(d2 - eps * eps) > 1e-12  # no tie at this seed
                if d2 < eps * eps:
                    arrivals += 1
                    exp = _goal_draw(seed, e, before.ep[e], i, before.t[e] + 1)
                    assert (s.gx[g], s.gy[g]) == exp
                else:
                    assert (s.gx[g], s.gy[g]) == (before.gx[g], before.gy[g])
            col = sum(1 for i, j in itertools.combinations(range(N), 2)
                      if (p1x[N * e + i] - p1x[N * e + j]) ** 2
                      + (p1y[N * e + i] - p1y[N * e + j]) ** 2 < 0.17 ** 2)
            assert abs(rew[e] - (d_rew - col)) < 1e-12
    assert arrivals >= E
    assert int(s.counters.reshape(E, 8)[:, oracle.CNT_SUCCESS].sum()) == arrivals


def test_waypoint_off_keeps_goals_and_rejects_foraging():
    N, E = 4, 16
    c = oracle.default_cfg(n_max=N, episode_len=10_000)
    s = oracle.reset(c, 3, [N] * E)
    g0 = (s.gx.copy(), s.gy.copy())
    for _ in range(300):
        oracle.step(c, 3, s)
    assert np.array_equal(s.gx, g0[0]) and np.array_equal(s.gy, g0[1])
    assert s.counters.reshape(E, 8)[:, oracle.CNT_SUCCESS].sum() == 0
    cf = oracle.default_cfg(oracle.FORAGE, n_max=N, goal_eps=0.05)
    with pytest.raises(Exception):
        oracle.reset(cf, 3, [N] * E)
