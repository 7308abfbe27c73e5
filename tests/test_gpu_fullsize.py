"""Parity at the full sizes of the benchmark's workloads, in the launch configuration the
benchmark times: the GPU batch is first driven into a random state by a scripted rollout, then
stepped a few times (the step selects the same kernels as the rollout: the 4-robot shuffle team
kernel in its spread launch, 6-7 envs per warp, for 4096 x 4; the per-class team kernels
otherwise), with the FP64 oracle stepped from the same states over the whole batch."""
import numpy as np
import pytest
import torch

import oracle
from pairing import make_pair, obs_diff, to_oracle_state, wrap

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2505_06771_gb300 as m
    m.lib()
    return m


@pytest.mark.parametrize("case", ["nav4096x4", "uneven8192", "largen1024x20"])
def test_full_size_teacher_forced(rl, case):
    from synth_inputs import uneven_robot_counts
    if case == "nav4096x4":
        g, o = make_pair(0, 4)
        n, warm = np.full(4096, 4, np.int32), 250
    elif case == "uneven8192":
        g, o = make_pair(1, 10)
        n, warm = uneven_robot_counts(0, 8192, 2, 10), 150
    else:
        g, o = make_pair(0, 20, near_frac=0.3)
        n, warm = np.full(1024, 20, np.int32), 60
    E, seed = len(n), 1000
    env = rl.Env(g, E, n, seed)
    R = env.total_robots
    env.rollout(warm)  # into a random state (no trajectory kept)
    obs = torch.empty(R, env.obs_dim, device="cuda")
    rew = torch.empty(E, device="cuda")
    done = torch.empty(E, dtype=torch.uint8, device="cuda")
    worst = dict(pose=0.0, th=0.0, rew=0.0, obs=0.0)
    for t in range(3):
        st = env.state_arrays()
        s = to_oracle_state(o, st)
        obs_o, rew_o, done_o, _ = oracle.step(o, seed, s)
        env.step(obs=obs, reward=rew, done=done)
        torch.cuda.synchronize()
        st2 = env.state_arrays()
        assert np.array_equal(done.cpu().numpy(), done_o)
        assert np.array_equal(st2["t"], s.t) and np.array_equal(st2["ep"], s.ep)
        cg, co = st2["counters"], s.counters.reshape(-1, 8)
        for c in (0, 1, 2, 6):
            assert np.array_equal(cg[:, c], co[:, c]), f"counter {c} at step {t}"
        if o["r_max"] > 0:
            assert np.array_equal(st2["qactive"], s.qactive)
        worst["pose"] = max(worst["pose"], np.abs(st2["x"] - s.x).max(), np.abs(st2["y"] - s.y).max())
        worst["th"] = max(worst["th"], np.abs(wrap(st2["th"] - s.th)).max())
        worst["rew"] = max(worst["rew"], np.abs(rew.cpu().numpy() - rew_o).max())
        worst["obs"] = max(worst["obs"], obs_diff(obs.cpu().numpy(), obs_o, g["scenario"],
                                                  g["n_max"], g["r_max"]))
    print(f"\n{case}: {E} envs, {R} robots, max errors {worst}")
    assert worst["pose"] < 1e-6 and worst["th"] < 1e-5
    assert worst["rew"] < 1e-5 and worst["obs"] < 1e-5
    env.close()
