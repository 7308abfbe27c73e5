"""Parity at the full sizes of the benchmark's workloads, in every launch shape the benchmark can
time.  The GPU batch is first driven into a random state by a scripted rollout; then it advances
through rl_rollout with T = 1 -- the benchmark's own call, its CUDA graph and the handle's launch
shape -- a few times, with the FP64 oracle stepped from the same states over the whole batch.

Launch shapes: every candidate the autotuner can pick for the 4096 x 4 batch (the shuffle and
gather team kernels with the spread launch or 2..8 envs per warp on a grid stride, the shuffle
kernel with its outputs in a second warp, one thread per env, two lanes per env), the shape the autotuner actually picks on this GPU, and for the
uneven batch the one persistent launch over every size class (the benchmark's launch) as well
as one launch per class.

Bars (binary32): done flags, step/episode counters, collision/out-of-arena/success counters and
resource states exact; poses within 3e-7 m per step, which is the control tolerance 1e-5 times
dt (a step error in the filtered velocity moves the projected point by dt times that error);
headings within 2e-5; rewards and observations within 1e-5."""
import numpy as np
import pytest
import torch

import oracle
from pairing import make_pair, obs_diff, to_oracle_state, wrap

pytestmark = pytest.mark.gpu

POSE_STEP_TOL = 3e-7  # 1e-5 (filtered control) x dt (0.033 s)


@pytest.fixture(scope="module")
def rl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2505_06771_gb300 as m
    m.lib()
    return m


def _candidates_4robot():
    """The autotuner's candidates for a 4-robot binary32 class (rl_tune)."""
    out = {}
    for var, name in ((1, "shuffle"), (2, "gather")):
        for we in (0, 2, 4, 6, 7, 8):
            out[f"{name}_we{we}"] = dict(lanes=4, block_threads=128, warp_envs=we, small_variant=var)
    out["split"] = dict(lanes=4, block_threads=128, warp_envs=0, small_variant=3)
    for we in (8, 16, 32):
        out[f"thread_we{we}"] = dict(lanes=1, block_threads=4 * we)
    out["lanes2"] = dict(lanes=2, block_threads=64)
    return out


SHAPES_4 = _candidates_4robot()


def _case(case):
    from synth_inputs import uneven_robot_counts
    if case == "nav4096x4":
        g, o = make_pair(0, 4)
        return g, o, np.full(4096, 4, np.int32), 250
    if case == "uneven8192":
        g, o = make_pair(1, 10)
        return g, o, uneven_robot_counts(0, 8192, 2, 10), 150
    g, o = make_pair(0, 20, near_frac=0.3)
    return g, o, np.full(1024, 20, np.int32), 60


def _run(rl, g, o, n, warm, tune=False, one_launch=None, steps=3, seed=1000):
    E = len(n)
    env = rl.Env(g, E, n, seed)
    choice = env.tune(50) if tune else None
    if one_launch is not None:
        env.set_class_launch(one_launch)
    R = env.total_robots
    env.rollout(warm)  # into a random state (no trajectory kept)
    obs = torch.empty(1, R, env.obs_dim, device="cuda")
    rew = torch.empty(1, E, device="cuda")
    done = torch.empty(1, E, dtype=torch.uint8, device="cuda")
    worst = dict(pose=0.0, th=0.0, rew=0.0, obs=0.0)
    for t in range(steps):
        st = env.state_arrays()
        s = to_oracle_state(o, st)
        obs_o, rew_o, done_o, _ = oracle.step(o, seed, s)
        env.rollout(1, obs, rew, done)  # the benchmark's call: graph replay of the tuned launch
        torch.cuda.synchronize()
        st2 = env.state_arrays()
        assert np.array_equal(done[0].cpu().numpy(), done_o), f"done differs at step {t}"
        assert np.array_equal(st2["t"], s.t) and np.array_equal(st2["ep"], s.ep)
        cg, co = st2["counters"], s.counters.reshape(-1, 8)
        for c in (0, 1, 2, 6):
            assert np.array_equal(cg[:, c], co[:, c]), f"counter {c} at step {t}"
        if o["r_max"] > 0:
            assert np.array_equal(st2["qactive"], s.qactive)
            assert np.array_equal(st2["qlevel"], s.qlevel)
        worst["pose"] = max(worst["pose"], np.abs(st2["x"] - s.x).max(), np.abs(st2["y"] - s.y).max())
        worst["th"] = max(worst["th"], np.abs(wrap(st2["th"] - s.th)).max())
        worst["rew"] = max(worst["rew"], np.abs(rew[0].cpu().numpy() - rew_o).max())
        worst["obs"] = max(worst["obs"], obs_diff(obs[0].cpu().numpy(), obs_o, g["scenario"],
                                                  g["n_max"], g["r_max"]))
    env.close()
    return worst, choice


def _check(worst):
    assert worst["pose"] < POSE_STEP_TOL and worst["th"] < 2e-5
    assert worst["rew"] < 1e-5 and worst["obs"] < 1e-5


@pytest.mark.parametrize("shape", list(SHAPES_4))
def test_nav4096x4_every_tuner_shape(rl, shape):
    g, o, n, warm = _case("nav4096x4")
    g.update(SHAPES_4[shape])
    worst, _ = _run(rl, g, o, n, warm)
    print(f"\nnav4096x4 {shape}: max errors {worst}")
    _check(worst)


@pytest.mark.parametrize("case", ["nav4096x4", "uneven8192", "largen1024x20"])
def test_full_size_tuned_launch(rl, case):
    """The launch shape the autotuner picks on this GPU (as the benchmark runs it)."""
    g, o, n, warm = _case(case)
    worst, choice = _run(rl, g, o, n, warm, tune=True)
    print(f"\n{case} tuned {choice}: max errors {worst}")
    _check(worst)


@pytest.mark.parametrize("one_launch", [1, 0, 2])
def test_uneven8192_one_launch_and_per_class(rl, one_launch):
    """The uneven batch through the one persistent launch over every size class (the kernel the
    uneven benchmark times) and through one launch per class, each against the oracle."""
    g, o, n, warm = _case("uneven8192")
    worst, _ = _run(rl, g, o, n, warm, one_launch=one_launch)
    print(f"\nuneven8192 one_launch={one_launch}: max errors {worst}")
    _check(worst)


def test_largen_default_launch(rl):
    g, o, n, warm = _case("largen1024x20")
    worst, _ = _run(rl, g, o, n, warm)
    print(f"\nlargen1024x20 default launch: max errors {worst}")
    _check(worst)
