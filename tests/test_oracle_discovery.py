"""Pins of the oracle's Discovery scenario (App. B "Discovery": sensing robots sense
landmarks within their sensing radius, tagging robots tag landmarks within their tagging
radius, rewards 1 per landmark sensed and 5 per landmark tagged, a 0.05 penalty per step while
a landmark is left to tag, no collision penalty; 4 robots, 2 of each role, radii 0.45 and
0.25, 100 steps).  CPU only: the rule is recomputed from dumped states by brute force."""
import numpy as np

import oracle


def _proj(s, l=0.05):
    return s.x + l * np.cos(s.th), s.y + l * np.sin(s.th)


def _wrap(a):
    return (a + np.pi) % (2 * np.pi) - np.pi


def test_roles_landmarks_and_full_length_episodes():
    N, E = 4, 64
    c = oracle.default_cfg(oracle.DISCOVERY, n_max=N)
    s = oracle.reset(c, 3, [N] * E)
    assert np.array_equal(s.level.reshape(E, N), np.tile([1, 1, 2, 2], (E, 1)))
    R = c["r_max"]
    assert np.all((s.n_res >= 2) & (s.n_res <= 6))
    for e in range(E):
        assert np.all(s.qlevel[R * e:R * e + s.n_res[e]] == 0)      # none sensed
        assert np.all(s.qactive[R * e:R * e + s.n_res[e]] == 1)     # all to tag
    s3 = oracle.reset(c, 3, [3] * 8)
    assert np.array_equal(s3.level.reshape(8, 3), np.tile([1, 1, 2], (8, 1)))
    for t in range(99):
        _, _, done, _ = oracle.step(c, 3, s)
        assert not done.any()
    _, _, done, _ = oracle.step(c, 3, s)
    assert done.all()


def test_transition_and_reward_by_brute_force():
    N, E, seed = 4, 96, 12
    c = oracle.default_cfg(oracle.DISCOVERY, n_max=N)
    s = oracle.reset(c, seed, [N] * E)
    R = c["r_max"]
    tagged_total = 0
    events = 0
    for t in range(99):
        before = s.copy()
        _, rew, _, _ = oracle.step(c, seed, s)
        px, py = _proj(s)
        for e in range(E):
            role = before.level[N * e:N * e + N]
            rsum = 0.0
            left = 0
            for k in range(before.n_res[e]):
                g = R * e + k
                d2 = (px[N * e:N * e + N] - before.qx[g]) ** 2 + (py[N * e:N * e + N] - before.qy[g]) ** 2
                sensed = bool(before.qlevel[g]) or bool(np.any((role == 1) & (d2 < 0.45 ** 2)))
                tagged = (not before.qactive[g]) or (sensed and bool(np.any((role == 2) & (d2 < 0.25 ** 2))))
                assert s.qlevel[g] == int(sensed) and s.qactive[g] == int(not tagged)
                if sensed and not before.qlevel[g]:
                    rsum += 1.0
                    events += 1
                if tagged and before.qactive[g]:
                    rsum += 5.0
                    tagged_total += 1
                    events += 1
                left += int(not tagged)
            if left > 0:
                rsum -= 0.05
            assert abs(rew[e] - rsum) < 1e-12
    assert events > 50 and tagged_total > 10
    assert int(s.counters.reshape(E, 8)[:, oracle.CNT_SUCCESS].sum()) == tagged_total


def test_observations_and_scripted_targets():
    N, E, seed = 4, 32, 5
    c = oracle.default_cfg(oracle.DISCOVERY, n_max=N, noise_amp=0.0)
    s = oracle.reset(c, seed, [N] * E)
    for _ in range(30):
        oracle.step(c, seed, s)
    before = s.copy()
    obs, _, _, tr = oracle.step(c, seed, s, trace=True)
    R = c["r_max"]
    od = 5 + 5 * (N - 1) + 4 * R
    assert obs.shape[1] == od
    xo, yo = 1.6 + 3.2, 1.0 + 2.0
    for e in range(E):
        for i in range(N):
            g = N * e + i
            o = obs[g]
            role = s.level[g]
            assert np.array_equal(o[:5], [s.x[g], s.y[g], s.th[g], 0.45 if role == 1 else 0.0,
                                          0.25 if role == 2 else 0.0])
            for slot, j in enumerate([j for j in range(N) if j != i]):
                gj = N * e + j
                q = o[5 + 5 * slot:10 + 5 * slot]
                assert abs(q[0] - (s.x[gj] - s.x[g])) < 1e-15 and abs(q[1] - (s.y[gj] - s.y[g])) < 1e-15
                assert abs(_wrap(q[2] - (s.th[gj] - s.th[g]))) < 1e-12
                assert q[3] == (0.45 if s.level[gj] == 1 else 0.0) and q[4] == (0.25 if s.level[gj] == 2 else 0.0)
            base = 5 + 5 * (N - 1)
            for k in range(R):
                q = o[base + 4 * k:base + 4 * k + 4]
                gk = R * e + k
                if k >= s.n_res[e]:
                    assert not q.any()
                elif s.qlevel[gk]:
                    assert np.allclose(q, [s.qx[gk] - s.x[g], s.qy[gk] - s.y[g], 1.0,
                                           1.0 - s.qactive[gk]], atol=1e-15, rtol=0)
                else:
                    assert np.allclose(q, [xo - s.x[g], yo - s.y[g], 0.0, 0.0], atol=1e-15, rtol=0)
    # scripted targets: sensing robots head for the nearest unsensed landmark, taggers for the
    # nearest sensed untagged one; without one, the nominal velocity is zero
    px, py = _proj(before)
    for e in range(E):
        for i in range(N):
            g = N * e + i
            ks = [k for k in range(before.n_res[e])
                  if (not before.qlevel[R * e + k]) if before.level[g] == 1] if before.level[g] == 1 else \
                 [k for k in range(before.n_res[e])
                  if before.qlevel[R * e + k] and before.qactive[R * e + k]]
            if not ks:
                assert np.all(tr["u_nom"][g] == 0.0)
                continue
            d2 = [(before.qx[R * e + k] - px[g]) ** 2 + (before.qy[R * e + k] - py[g]) ** 2 for k in ks]
            k = ks[int(np.argmin(d2))]
            v = np.array([before.qx[R * e + k] - px[g], before.qy[R * e + k] - py[g]])
            n = np.hypot(*v)
            if n > 0.2:
                v *= 0.2 / n
            assert np.allclose(tr["u_nom"][g], v, atol=1e-15, rtol=0)


def test_monotone_flags_over_rollouts():
    N, E = 6, 40
    c = oracle.default_cfg(oracle.DISCOVERY, n_max=N, episode_len=1000)
    s = oracle.reset(c, 9, [N] * E)
    R = c["r_max"]
    live = (np.arange(R)[None, :] < s.n_res[:, None]).reshape(-1)  # landmark slots in use
    prev = s.copy()
    for _ in range(200):
        oracle.step(c, 9, s)
        assert np.all(s.qlevel >= prev.qlevel)                 # sensed stays sensed
        assert np.all(s.qactive <= prev.qactive)               # tagged stays tagged
        assert np.all(((s.qactive == 1) | (s.qlevel == 1))[live])  # tagged implies sensed
        prev = s.copy()
