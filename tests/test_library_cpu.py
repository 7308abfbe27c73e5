"""CPU checks of the CUDA library: it builds for sm_103a, loads, exports every function that
include/rl.h declares, and its defaults agree with the oracle's constants.  No CUDA calls."""
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
