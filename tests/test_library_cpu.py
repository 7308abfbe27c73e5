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
