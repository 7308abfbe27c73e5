"""Pins of the oracle's random-number layer and reset sampler (CPU only).

Philox4x32-10 is checked against the published known-answer vectors; the sampler against the
properties its definition fixes (region, separation, near-pair share and distance, levels)
and against a recomputation from the pinned generator.
"""
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert [int(v) for v in oracle.philox4x32_10(ctr, key)] == out


def _u01(w):
    return np.float32(np.uint32(w) >> np.uint32(8)) * np.float32(2.0 ** -24)


def test_sampler_first_robot_recomputed_from_generator():
    c = oracle.default_cfg(n_max=4)
    seed = 0x1234_5678_9ABC
    s = oracle.reset(c, seed, [4] * 8)
    f32 = np.float32
    lox = f32(-1.6) + f32(0.2)
    hix = f32(1.6) - f32(0.2)
    loy = f32(-1.0) + f32(0.2)
    hiy = f32(1.0) - f32(0.2)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for e in range(8):
        w = oracle.philox4x32_10([e, 0, (2 << 24) | 0, 0], key)
        x0 = lox + _u01(w[0]) * (hix - lox)
        y0 = loy + _u01(w[1]) * (hiy - loy)
        th0 = -f32(np.pi) + _u01(w[2]) * f32(2 * np.pi)
        assert s.x[4 * e] == float(x0) and s.y[4 * e] == float(y0) and s.th[4 * e] == float(th0)
        wg = oracle.philox4x32_10([e, 0, (3 << 24) | 2, 0], key)
        assert s.gx[4 * e + 2] == float(lox + _u01(wg[0]) * (hix - lox))
        assert s.gy[4 * e + 2] == float(loy + _u01(wg[1]) * (hiy - loy))


@pytest.mark.parametrize("N", [2, 4, 12, 20])
def test_sampler_region_and_separation(N):
    c = oracle.default_cfg(n_max=N)
    E = 256
    s = oracle.reset(c, 7, [N] * E)
    x = s.x.reshape(E, N).astype(np.float32)
    y = s.y.reshape(E, N).astype(np.float32)
    assert np.all(s.x >= -1.4 - 1e-6) and np.all(s.x <= 1.4 + 1e-6)
    assert np.all(s.y >= -0.8 - 1e-6) and np.all(s.y <= 0.8 + 1e-6)
    assert np.all(s.gx >= -1.4 - 1e-6) and np.all(s.gx <= 1.4 + 1e-6)
    assert np.all(np.abs(s.th) <= np.float32(np.pi))
    dx = x[:, :, None] - x[:, None, :]
    dy = y[:, :, None] - y[:, None, :]
    d2 = dx * dx + dy * dy + np.eye(N, dtype=np.float32) * 9
    assert d2.min() >= np.float32(0.3) * np.float32(0.3)
    # projected points of a safe start are at least 0.3 - 2 l = 0.2 > r apart
    px = s.x + 0.05 * np.cos(s.th)
    py = s.y + 0.05 * np.sin(s.th)
    P, Q = px.reshape(E, N), py.reshape(E, N)
    dp = np.sqrt((P[:, :, None] - P[:, None, :]) ** 2 + (Q[:, :, None] - Q[:, None, :]) ** 2)
    assert (dp + 9 * np.eye(N)).min() >= 0.2 - 1e-6


def test_sampler_near_pairs():
    N, E = 20, 2000
    c = oracle.default_cfg(n_max=N, near_frac=0.3)
    s = oracle.reset(c, 3, [N] * E)
    x, y, th = s.x.reshape(E, N), s.y.reshape(E, N), s.th.reshape(E, N)
    d01 = np.hypot(x[:, 0] - x[:, 1], y[:, 0] - y[:, 1])
    near = d01 < 0.25
    frac = near.mean()
    # binomial(2000, 0.3): 6 sigma band
    assert abs(frac - 0.3) < 6 * np.sqrt(0.3 * 0.7 / E)
    assert np.all(d01[near] >= 0.18 - 1e-6) and np.all(d01[near] <= 0.20 + 1e-6)
    assert np.all(th[near, 0] == th[near, 1])
    # h = d^2 - r^2 of the projected points is small and positive
    px, py = x + 0.05 * np.cos(th), y + 0.05 * np.sin(th)
    h = (px[near, 0] - px[near, 1]) ** 2 + (py[near, 0] - py[near, 1]) ** 2 - 0.17 ** 2
    assert np.all(h > 0.0034) and np.all(h < 0.0112)
    # the other robots keep the 0.3 m separation from the near pair
    for e in np.nonzero(near)[0][:50]:
        d = np.hypot(x[e, 2:, None] - x[e, None, :2], y[e, 2:, None] - y[e, None, :2])
        assert d.min() >= 0.3 - 1e-6


def test_sampler_foraging_levels_and_resources():
    c = oracle.default_cfg(oracle.FORAGE, n_max=10)
    E = 3000
    n = np.random.default_rng(0).integers(2, 11, E).astype(np.int32)
    s = oracle.reset(c, 11, n)
    assert set(np.unique(s.level)) == {1, 2, 3}
    assert s.n_res.min() == 2 and s.n_res.max() == 6
    counts = np.bincount(s.n_res, minlength=7)[2:]
    assert np.all(np.abs(counts / E - 0.2) < 0.04)
    ql = s.qlevel.reshape(E, 6)
    qa = s.qactive.reshape(E, 6)
    for e in range(E):
        k = s.n_res[e]
        assert np.all(qa[e, :k] == 1) and np.all(qa[e, k:] == 0)
        assert np.all((ql[e, :k] >= 1) & (ql[e, :k] <= 3))


def test_reset_is_a_function_of_seed_env_episode():
    c = oracle.default_cfg(n_max=4)
    a = oracle.reset(c, 5, [4] * 6)
    b = oracle.reset(c, 5, [4] * 6)
    d = oracle.reset(c, 6, [4] * 6)
    e = oracle.reset(c, 5, [4] * 6, ep=[1] * 6)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.th, b.th)
    assert not np.array_equal(a.x, d.x)
    assert not np.array_equal(a.x, e.x)
