"""CPU checks of the CUDA library: it builds for sm_103a, loads, exports every function that
include/rl.h declares, its defaults agree with the oracle's constants, and its calls reject
invalid configurations, robot counts and null handles with RL_ERR_ARG before any CUDA call.  No
CUDA calls."""
import ctypes

import pytest

import oracle


@pytest.fixture(scope="module")
def rl():
    import paper_2505_06771_gb300 as m
    m.build()
    return m


def test_exports_every_declared_symbol(rl):
    L = rl.lib()
    names = rl.exported_symbols()
    assert "rl_create" in names and "rl_step" in names and "rl_rollout" in names
    for n in names:
        assert hasattr(L, n), n


def test_defaults_agree_with_oracle(rl):
    for scen in (rl.NAVIGATION, rl.FORAGING):
        g = rl.config_default(scen)
        o = oracle.default_cfg(scen)
        for k in ("gamma", "r", "l", "vmax", "wmax", "dt", "kappa", "k_si", "noise_amp", "c_col",
                  "forage_radius", "xmin", "xmax", "ymin", "ymax", "init_margin", "min_sep",
                  "episode_len", "n_res_min", "n_res_max", "r_max", "max_attempts"):
            assert g[k] == o[k], (scen, k)
    assert rl.lib().rl_config_default(7, ctypes.byref(rl.RLConfig())) == 1


def test_state_blob_parser_layout():
    import numpy as np
    import paper_2505_06771_gb300 as m
    # header + image of 17 segments for E=2 envs, 5 robots, binary32, no resources
    E, T = 2, 5
    lens = [T * 4] * 5 + [T * 4, E * 4, E * 4, E * 4, 0, 0, 0, 0, E * 32, E * 4, (E + 1) * 4,
                          T * 4]
    img = b"".join(bytes([i + 1]) * n + b"\0" * (((n + 255) & ~255) - n) for i, n in enumerate(lens))
    hdr = np.array([0x31534C52, 2, 32, 0, E, T, 0, 3], np.int32).tobytes()
    hdr += np.array([7, len(img)], np.uint64).tobytes() + b"\0" * 16
    st = m.parse_state(hdr + img)
    assert st["n_envs"] == 2 and st["seed"] == 7
    assert st["x"].view(np.uint8)[0] == 1 and st["off"].view(np.uint8)[0] == 16
    assert st["gth"].view(np.uint8)[0] == 17 and len(st["gth"]) == T


def test_every_declaration_is_documented():
    """Each function include/rl.h declares carries a comment of its own: a block comment ending
    on the line before its declaration (or before the group of declarations it heads), or one
    on the declaration's own line."""
    import os
    import re
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                       "rl.h")
    lines = open(hdr).read().splitlines()
    decl = re.compile(r"^\s*(?:rl_status|size_t|int32_t|const char\*|void)\s+(rl_[a-z_0-9]+)\s*\(")
    seen = []
    for i, ln in enumerate(lines):
        m = decl.match(ln)
        if not m:
            continue
        seen.append(m.group(1))
        if "/*" in ln:
            continue
        j = i - 1
        # a group of declarations under one comment, or a declaration continued over lines
        while j >= 0 and (decl.match(lines[j]) or lines[j].startswith(" " * 8) or
                          lines[j].strip().startswith("#define")):
            j -= 1
        assert j >= 0 and lines[j].rstrip().endswith("*/"), f"{m.group(1)} has no comment"
    assert set(seen) >= {"rl_create", "rl_reset", "rl_step", "rl_rollout", "rl_destroy",
                         "rl_rollout_noalloc", "rl_set_class_launch"}


def test_boundary_calls_cite_the_paper():
    """The calls that restate a step of the method name the passage they follow."""
    import os
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "include", "rl.h")).read()
    for name, passage in (("rl_create", "Sec. 6.1"), ("rl_reset", "Sec. 6.1"),
                          ("rl_step", "Dec-POMDP"), ("rl_rollout", "Sec. 4.1"),
                          ("rl_policy_create", "App. A")):
        k = hdr.index(f"rl_status {name}(")
        comment = hdr[hdr.rindex("/*", 0, k):k]
        assert passage in comment or passage in hdr[:hdr.index("#ifndef")], (name, passage)


# Configurations rl_create rejects with RL_ERR_ARG before any CUDA call (so they run without a
# GPU): each override breaks one rule of the configuration check.
BAD_CONFIGS = [
    (0, dict(scenario=7)), (0, dict(precision=16)), (0, dict(episode_len=0)),
    (0, dict(max_attempts=0)), (0, dict(l=0.0)), (0, dict(vmax=-0.2)), (0, dict(wmax=0.0)),
    (0, dict(dt=0.0)), (0, dict(r=-0.1)), (0, dict(xmax=-2.0)), (0, dict(ymax=-2.0)),
    (0, dict(n_max=33)), (0, dict(n_max=-1)), (0, dict(block_threads=48)),
    (0, dict(block_threads=512)), (0, dict(lanes=-1)), (0, dict(warp_envs=-1)),
    (0, dict(goal_eps=-0.1)), (0, dict(controller=5)),
    (0, dict(controller=1, pose_k1=0.0)),
    (1, dict(r_max=0)), (1, dict(r_max=17)), (1, dict(n_res_min=3, n_res_max=2)),
    (1, dict(n_res_max=99)), (1, dict(goal_eps=0.1)), (1, dict(controller=1)),
]


def _create(rl, cfg, n_envs, n_robots_uniform=4, per_env=None):
    h = ctypes.c_void_p()
    arr = None
    if per_env is not None:
        import numpy as np
        arr = np.ascontiguousarray(per_env, dtype=np.int32)
    st = rl.lib().rl_create(ctypes.byref(rl._to_struct(cfg)), n_envs,
                            None if arr is None else arr.ctypes.data, n_robots_uniform, 0,
                            None, ctypes.byref(h))
    return st, h.value


@pytest.mark.parametrize("scen,override", BAD_CONFIGS)
def test_create_rejects_each_invalid_configuration(rl, scen, override):
    g = rl.config_default(scen)
    g.update(override)
    st, h = _create(rl, g, 4)
    assert st == 1 and h is None, (override, st)


@pytest.mark.parametrize("n_envs,uniform,per_env,n_max", [
    (0, 4, None, 0),                 # no envs
    (4, 0, None, 0),                 # no robots
    (4, 33, None, 0),                # more robots than a team holds
    (3, 0, [4, 0, 2], 0),            # one env without robots
    (3, 0, [4, 33, 2], 0),           # one env over the limit
    (3, 0, [4, 6, 2], 4),            # n_max below the largest env
])
def test_create_rejects_robot_counts(rl, n_envs, uniform, per_env, n_max):
    g = rl.config_default(rl.NAVIGATION, n_max=n_max)
    st, h = _create(rl, g, n_envs, uniform, per_env)
    assert st == 1 and h is None


def test_calls_on_a_null_handle_are_argument_errors(rl):
    L = rl.lib()
    assert L.rl_step(None, None, None, None, None) == 1
    assert L.rl_rollout(None, 10, None, None, None) == 1
    assert L.rl_rollout_plain(None, 10, None, None, None) == 1
    assert L.rl_rollout_host(None, None, 10, None, None, None) == 1
    assert L.rl_sync(None) == 1
    assert L.rl_obs_dim(None) == 0 and L.rl_n_envs(None) == 0 and L.rl_total_robots(None) == 0
    assert L.rl_last_error(None) == b"null handle"
    L.rl_destroy(None)  # a no-op
