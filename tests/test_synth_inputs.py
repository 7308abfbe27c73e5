"""The seeded input generators against the recipes they implement (CPU): ranges, distributions,
shapes and determinism.  They feed both the oracle and the CUDA path, so a drift here would move
both sides together and no parity test would see it."""
import numpy as np

import synth_inputs as si


def test_uneven_robot_counts_uniform_over_the_range():
    n = si.uneven_robot_counts(0, 8192)
    assert n.dtype == np.int32 and n.shape == (8192,)
    assert n.min() == 2 and n.max() == 10
    counts = np.bincount(n, minlength=11)[2:]
    # uniform over 9 values: each count within 5 standard deviations of 8192 / 9
    mean, sd = 8192 / 9, np.sqrt(8192 * (1 / 9) * (8 / 9))
    assert np.all(np.abs(counts - mean) < 5 * sd)
    assert np.array_equal(n, si.uneven_robot_counts(0, 8192))
    assert not np.array_equal(n, si.uneven_robot_counts(1, 8192))
    assert set(si.uneven_robot_counts(3, 500, 1, 10)) == set(range(1, 11))


def test_policy_actions_bounded_and_keyed_by_seed_and_step():
    a = si.policy_actions(5, 0, 1000)
    assert a.shape == (1000, 2) and a.dtype == np.float32
    assert np.abs(a).max() <= 0.3 and np.abs(a).max() > 0.29
    assert abs(float(a.mean())) < 0.02
    assert np.array_equal(a, si.policy_actions(5, 0, 1000))
    assert not np.array_equal(a, si.policy_actions(5, 1, 1000))
    assert not np.array_equal(a, si.policy_actions(6, 0, 1000))
    assert si.policy_actions(5, 0, 10, dtype=np.float64).dtype == np.float64


def test_policy_weights_shapes_and_fan_in_bounds():
    H, od = 128, 12
    w = si.policy_weights(7, H, od)
    shapes = dict(w1=(H, od), b1=(H,), wi=(3 * H, H), bi=(3 * H,), wh=(3 * H, H), bh=(3 * H,),
                  wo=(2, H), bo=(2,))
    assert {k: v.shape for k, v in w.items()} == shapes
    assert all(v.dtype == np.float32 for v in w.values())
    assert np.abs(w["w1"]).max() <= 1 / np.sqrt(od) and np.abs(w["b1"]).max() <= 1 / np.sqrt(od)
    for k in ("wi", "bi", "wh", "bh", "wo"):
        assert np.abs(w[k]).max() <= 1 / np.sqrt(H) + 1e-7, k
        assert np.abs(w[k]).max() > 0.9 / np.sqrt(H), k
    assert np.abs(w["bo"]).max() <= 0.1
    w2 = si.policy_weights(7, H, od)
    assert all(np.array_equal(w[k], w2[k]) for k in w)


def test_serving_requests_poisson_arrivals_and_ranges():
    dur, rate = 20.0, 200.0
    reqs = si.serving_requests(100, dur, rate_hz=rate)
    n = len(reqs)
    # Poisson count: within 5 standard deviations of rate x duration
    assert abs(n - rate * dur) < 5 * np.sqrt(rate * dur)
    t = np.array([r["arrival_s"] for r in reqs])
    assert np.all(np.diff(t) > 0) and t[0] > 0 and t[-1] < dur
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / rate) < 0.1 / rate
    # exponential gaps: the standard deviation equals the mean
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1
    e = np.array([r["n_envs"] for r in reqs])
    assert e.min() >= 1 and e.max() <= 2048
    # log-uniform on [1, 2048]: the median of ln(n) near ln(2048) / 2
    assert abs(np.median(np.log(e + 0.5)) - np.log(2048) / 2) < 0.3
    rob = np.array([r["n_robots"] for r in reqs])
    assert rob.min() == 2 and rob.max() == 12
    hor = np.array([r["horizon"] for r in reqs])
    assert hor.min() >= 100 and hor.max() <= 1000
    assert [r["id"] for r in reqs] == list(range(n))
    assert len({r["seed"] for r in reqs}) == n
    assert reqs == si.serving_requests(100, dur, rate_hz=rate)
