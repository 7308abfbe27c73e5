"""Policy in the loop (GPU): a one-layer MLP -> GRU -> linear policy (App. A's shape) evaluated
on the device between steps, against a float64 numpy forward that applies the same bf16
roundings (inputs, first-layer weights and bias, GRU weights, the previous state fed to the
GEMM) and the same per-robot state reset at episode ends."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2505_06771_gb300 as m
    m.lib()
    return m


def _bf16(a):
    """Round to bf16 (nearest, ties to even) and back to float64."""
    b = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _weights(H, od, seed):
    g = np.random.default_rng(seed)
    s1, s2 = 1.0 / np.sqrt(od), 1.0 / np.sqrt(H)
    return dict(w1=g.uniform(-s1, s1, (H, od)), b1=g.uniform(-s1, s1, H),
                wi=g.uniform(-s2, s2, (3 * H, H)), bi=g.uniform(-s2, s2, 3 * H),
                wh=g.uniform(-s2, s2, (3 * H, H)), bh=g.uniform(-s2, s2, 3 * H),
                wo=g.uniform(-s2, s2, (2, H)), bo=g.uniform(-0.1, 0.1, 2))


def _reference(w, obs_seq, done_seq, rows, row_env, vmax):
    """Actions of every step from the observations feeding them (float64, bf16 where the GPU
    rounds)."""
    H = w["b1"].shape[0]
    w = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in w.items()}
    W1, B1 = _bf16(w["w1"]), _bf16(w["b1"])
    Wi, Wh = _bf16(w["wi"]), _bf16(w["wh"])
    h = np.zeros((rows, H))
    acts = []
    for t, o in enumerate(obs_seq):
        if t > 0:
            h[done_seq[t - 1][row_env].astype(bool)] = 0.0
        x = _bf16(o)
        h1 = _bf16(np.maximum(x @ W1.T + B1, 0.0))
        hb = _bf16(h)
        gi = h1 @ Wi.T + w["bi"]
        gh = hb @ Wh.T + w["bh"]
        r = 1 / (1 + np.exp(-(gi[:, :H] + gh[:, :H])))
        z = 1 / (1 + np.exp(-(gi[:, H:2 * H] + gh[:, H:2 * H])))
        n = np.tanh(gi[:, 2 * H:] + r * gh[:, 2 * H:])
        h = (1 - z) * n + z * h
        acts.append(vmax * np.tanh(h @ w["wo"].T + w["bo"]))
    return np.stack(acts)


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


@pytest.mark.parametrize("H,N,ep_len", [(128, 4, 100), (256, 3, 4)])
def test_policy_rollout_matches_reference_and_env(rl, H, N, ep_len):
    E, T = 96, 9
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
    ref = _reference(w, obs_seq, done.cpu().numpy(), R, row_env, g["vmax"])
    d = np.abs(act.cpu().numpy() - ref)
    print(f"\npolicy H={H}: action error max {d.max():.3e} mean {d.mean():.3e}; "
          f"episode ends {int(done.sum())}")
    if ep_len < T:
        assert done.cpu().numpy().any()
    assert d.max() < 5e-3 and d.mean() < 2e-4
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
