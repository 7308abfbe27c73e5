"""Shared test helpers: one configuration handed to both sides, and the GPU state blob turned
into an oracle State (inputs only -- no arithmetic of the method lives here)."""
import numpy as np

import oracle

SHARED = ("scenario", "scripted", "episode_len", "n_res_min", "n_res_max", "max_attempts",
          "r_max", "gamma", "r", "l", "vmax", "wmax", "dt", "kappa", "k_si", "noise_amp",
          "c_col", "forage_radius", "xmin", "xmax", "ymin", "ymax", "init_margin", "min_sep",
          "near_frac", "near_dmin", "near_dmax")


def make_pair(scenario, n_max, precision=32, **kw):
    """(gpu_cfg, oracle_cfg) with the same constants; overrides apply to both."""
    import paper_2505_06771_gb300 as rl
    g = rl.config_default(scenario)
    o = oracle.default_cfg(scenario, n_max=n_max)
    g["precision"] = precision
    g["n_max"] = n_max
    for k, v in kw.items():
        if k in g:
            g[k] = v
        if k in o:
            o[k] = v
    return g, o


def to_oracle_state(ocfg, st):
    """oracle.State from a parsed GPU state blob (values widened to double exactly)."""
    s = oracle.State(ocfg, st["n_robots"])
    for k in ("x", "y", "th", "gx", "gy", "gth"):
        getattr(s, k)[:] = st[k].astype(np.float64)
    s.level[:] = st["level"]
    s.t[:] = st["t"]
    s.ep[:] = st["ep"]
    s.n_res[:] = st["n_res"]
    R = st["r_max"]
    if R > 0:
        s.qx[:] = st["qx"].astype(np.float64)
        s.qy[:] = st["qy"].astype(np.float64)
        s.qlevel[:] = st["qlevel"]
        s.qactive[:] = st["qactive"]
    s.counters[:] = st["counters"].reshape(-1)
    return s


def wrap(a):
    return (np.asarray(a) + np.pi) % (2 * np.pi) - np.pi


def obs_angle_columns(scenario, n_max, r_max):
    """Observation columns that hold angles (compared modulo 2 pi)."""
    if scenario == 0:
        return [2] + [5 + 3 * s + 2 for s in range(n_max - 1)]
    if scenario == 2:
        return [2] + [5 + 5 * s + 2 for s in range(n_max - 1)]
    return [2] + [4 + 4 * s + 2 for s in range(n_max - 1)]


def obs_diff(a, b, scenario, n_max, r_max):
    """Max abs difference of two observation arrays, angles compared on the circle."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    d = np.abs(a - b)
    for c in obs_angle_columns(scenario, n_max, r_max):
        d[..., c] = np.abs(wrap(a[..., c] - b[..., c]))
    return float(d.max()) if d.size else 0.0
