"""rl_rollout_noalloc: the allocation-free rollout (GPU).

Some callers cannot allocate device memory (another component owns the allocator, or a fixed
memory budget is enforced), so the library offers one rollout entry point whose environment
state lives in a static device array.  It must give the same trajectories as the handle-based
entry point (rl_create + rl_rollout), on two calls in a row: the array keeps the previous
call's contents, which must not leak into the next result.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-6  # binary32 trajectories; the same kernels run, so the match is expected bit for bit


@pytest.fixture(scope="module")
def rl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2505_06771_gb300 as m
    m.build()
    return m


def _buffers(T, rows, od, E, dt=torch.float32):
    return (torch.full((T, rows, od), 7.0, dtype=dt, device="cuda"),
            torch.full((T, E), 7.0, dtype=dt, device="cuda"),
            torch.full((T, E), 7, dtype=torch.uint8, device="cuda"))


# (scenario, robots, envs, steps, overrides).  The cases run in this order, so the Discovery case
# (r_max 4) lays its resource segments over the Foraging case's (r_max 6) at shifted offsets,
# the binary64 case reuses the array with 8-byte reals, and the last case takes a launch shape
# of its own (the shuffle team kernel, 8 envs per warp, grid stride) from the configuration.
CASES = [(0, 4, 1024, 150, {}), (1, 6, 300, 120, {}), (2, 5, 257, 110, dict(r_max=4, n_res_max=4)),
         (0, 4, 200, 100, dict(precision=64)), (0, 4, 600, 60, dict(block_threads=128, warp_envs=8, small_variant=1))]


@pytest.mark.parametrize("scenario,N,E,T,kw", CASES)
def test_noalloc_matches_handle_rollout_twice(rl, scenario, N, E, T, kw):
    g = rl.config_default(scenario, **kw)
    seeds = [11, 12]
    for call, seed in enumerate(seeds):
        env = rl.Env(g, E, N, seed)
        dt = env.dtype
        ro, rr, rd = _buffers(T, E * N, env.obs_dim, E, dt)
        env.rollout(T, ro, rr, rd)
        no, nr, nd = _buffers(T, E * N, env.obs_dim, E, dt)
        rl.rollout_noalloc(g, E, N, seed, T, no, nr, nd)
        torch.cuda.synchronize()
        assert (no - ro).abs().max().item() <= TOL, f"call {call}: observations differ"
        assert (nr - rr).abs().max().item() <= TOL, f"call {call}: rewards differ"
        assert torch.equal(nd, rd), f"call {call}: done flags differ"
        env.close()


def test_noalloc_rejects_oversized_batches(rl):
    g = rl.config_default(0)
    L = rl.lib()
    limit = rl.noalloc_max_bytes()
    assert rl.noalloc_state_bytes(g, 4096, 4) <= limit
    E = 1 << 20
    assert rl.noalloc_state_bytes(g, E, 4) > limit
    st = L.rl_rollout_noalloc(ctypes.byref(rl._to_struct(g)), E, 4, 0, 10, None, None, None, None)
    assert st == 1  # RL_ERR_ARG, before any GPU work
