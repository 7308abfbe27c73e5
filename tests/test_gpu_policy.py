"""Policy in the loop (GPU): a one-layer MLP -> GRU -> linear policy (App. A's shape) evaluated
on the device between steps, against the FP64 policy reference (oracle/policy.py) with the bf16
roundings of the tensor-core operands (inputs, first-layer weights and bias, GRU weights, the
previous state fed to the product) and the same per-robot state reset at episode ends.

Tolerance on actions: 5e-5 (|a| <= v_max = 0.2).  The GPU evaluates the gates' sigma and tanh
with the hardware tanh approximation (relative error about 2^-11) and accumulates the products
in binary32; the reference is exact in float64 apart from the stated bf16 roundings."""
import numpy as np
import pytest
import torch

from oracle.policy import policy_actions

ACT_TOL = 5e-5

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2505_06771_gb300 as m
    m.lib()
    return m


def _weights(H, od, seed):
    g = np.random.default_rng(seed)
    s1, s2 = 1.0 / np.sqrt(od), 1.0 / np.sqrt(H)
    return dict(w1=g.uniform(-s1, s1, (H, od)), b1=g.uniform(-s1, s1, H),
                wi=g.uniform(-s2, s2, (3 * H, H)), bi=g.uniform(-s2, s2, 3 * H),
                wh=g.uniform(-s2, s2, (3 * H, H)), bh=g.uniform(-s2, s2, 3 * H),
                wo=g.uniform(-s2, s2, (2, H)), bo=g.uniform(-0.1, 0.1, 2))


def test_observe_matches_the_step_observation(rl):
    g = rl.config_default(0, scripted=0, n_max=4)
    env = rl.Env(g, 33, 4, 7)
    R = env.total_robots
    obs = torch.zeros(R, env.obs_dim, device="cuda")
    rew = torch.zeros(33, device="cuda")
    done = torch.zeros(33, dtype=torch.uint8, device="cuda")
    env.step(actions=torch.full((R, 2), 0.05, device="cuda"), obs=obs, reward=rew, done=done)
    o2 = torch.full_like(obs, 7.0)
    env.observe(o2)
    torch.cuda.synchronize()
    assert torch.equal(obs, o2)
    env.close()


# H = 512 streams A's chunks through the stage ring (beyond the resident size) over four unit
# blocks; the full batch (4096 envs) runs the policy kernel on 128 tiles.
@pytest.mark.parametrize("H,N,ep_len,E", [(128, 4, 100, 96), (256, 3, 4, 96), (512, 4, 4, 96),
                                           (128, 4, 4, 4096)])
def test_policy_rollout_matches_reference_and_env(rl, H, N, ep_len, E):
    T = 9
    g = rl.config_default(0, scripted=0, n_max=N, episode_len=ep_len)
    env = rl.Env(g, E, N, 11)
    R, od = env.total_robots, env.obs_dim
    w = {k: v.astype(np.float32) for k, v in _weights(H, od, 3).items()}
    pol = rl.Policy(env, w)
    obs0 = torch.zeros(R, od, device="cuda")
    env.observe(obs0)
    obs = torch.zeros(T, R, od, device="cuda")
    done = torch.zeros(T, E, dtype=torch.uint8, device="cuda")
    rew = torch.zeros(T, E, device="cuda")
    act = torch.zeros(T, R, 2, device="cuda")
    # a twin handle stepped by hand with the policy's actions
    twin = rl.Env(g, E, N, 11)
    pol.rollout(T, obs0, obs, done, reward=rew, actions=act)
    torch.cuda.synchronize()
    for t in range(T):
        o = torch.zeros(R, od, device="cuda")
        rr = torch.zeros(E, device="cuda")
        dd = torch.zeros(E, dtype=torch.uint8, device="cuda")
        twin.step(actions=act[t].contiguous(), obs=o, reward=rr, done=dd)
        assert torch.equal(o, obs[t]) and torch.equal(dd, done[t]) and torch.equal(rr, rew[t])
    row_env = np.repeat(np.arange(E), N)
    obs_seq = [obs0.cpu().numpy()] + [obs[t].cpu().numpy() for t in range(T - 1)]
    w64 = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in w.items()}
    ref = policy_actions(w64, obs_seq, done.cpu().numpy(), row_env, g["vmax"], bf16=True)
    d = np.abs(act.cpu().numpy() - ref)
    print(f"\npolicy H={H}: action error max {d.max():.3e} mean {d.mean():.3e}; "
          f"episode ends {int(done.sum())}")
    if ep_len < T:
        assert done.cpu().numpy().any()
    assert d.max() < ACT_TOL
    # a second rollout continues the recurrent state; reset_hidden restarts it
    pol.reset_hidden()
    pol.close()
    twin.close()
    env.close()


def test_policy_arguments(rl):
    g = rl.config_default(0, n_max=4)  # scripted handle: no policy
    env = rl.Env(g, 8, 4, 1)
    with pytest.raises(rl.RLError):
        rl.Policy(env, {k: v.astype(np.float32) for k, v in _weights(128, env.obs_dim, 0).items()})
    env.close()
    g = rl.config_default(0, scripted=0, n_max=4)
    env = rl.Env(g, 8, 4, 1)
    with pytest.raises(rl.RLError):
        rl.Policy(env, {k: v.astype(np.float32) for k, v in _weights(100, env.obs_dim, 0).items()})
    env.close()
