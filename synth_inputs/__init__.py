"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

Only input generation lives here (robot counts per environment, policy actions, serving
request streams); none of the environment step's arithmetic.  Every generator is a numpy
PCG64 stream keyed by an explicit seed.
"""
from __future__ import annotations

import numpy as np


def uneven_robot_counts(seed: int, n_envs: int, lo: int = 2, hi: int = 10) -> np.ndarray:
    """Robot count per environment, uniform in {lo, ..., hi}."""
    return np.random.default_rng(seed).integers(lo, hi + 1, n_envs).astype(np.int32)


def policy_actions(seed: int, step: int, total_robots: int, amp: float = 0.3,
                   dtype=np.float32) -> np.ndarray:
    """Random SI velocity commands [total_robots, 2], uniform in [-amp, amp]^2."""
    rng = np.random.default_rng([seed, step])
    return rng.uniform(-amp, amp, (total_robots, 2)).astype(dtype)


def policy_weights(seed: int, hidden: int, obs_dim: int) -> dict:
    """Weights of the MLP -> GRU -> linear policy, each layer uniform in +-1/sqrt(fan_in)."""
    g = np.random.default_rng(seed)
    s1, s2 = 1.0 / np.sqrt(obs_dim), 1.0 / np.sqrt(hidden)
    H = hidden
    w = dict(w1=g.uniform(-s1, s1, (H, obs_dim)), b1=g.uniform(-s1, s1, H),
             wi=g.uniform(-s2, s2, (3 * H, H)), bi=g.uniform(-s2, s2, 3 * H),
             wh=g.uniform(-s2, s2, (3 * H, H)), bh=g.uniform(-s2, s2, 3 * H),
             wo=g.uniform(-s2, s2, (2, H)), bo=g.uniform(-0.1, 0.1, 2))
    return {k: v.astype(np.float32) for k, v in w.items()}


def serving_requests(seed: int, duration_s: float, rate_hz: float = 200.0,
                     envs_max: int = 2048, robots_lo: int = 2, robots_hi: int = 12,
                     horizon_lo: int = 100, horizon_hi: int = 1000) -> list[dict]:
    """Poisson arrivals of rollout requests: n_envs log-uniform in [1, envs_max], robots uniform
    in {robots_lo..robots_hi}, horizon uniform in {horizon_lo..horizon_hi}."""
    rng = np.random.default_rng(seed)
    out, t, k = [], 0.0, 0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        n_envs = int(np.floor(np.exp(rng.uniform(0.0, np.log(envs_max)))))
        out.append(dict(id=k, arrival_s=t, n_envs=max(1, min(envs_max, n_envs)),
                        n_robots=int(rng.integers(robots_lo, robots_hi + 1)),
                        horizon=int(rng.integers(horizon_lo, horizon_hi + 1)),
                        seed=int(rng.integers(0, 2 ** 63 - 1))))
        k += 1
    return out
