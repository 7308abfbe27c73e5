"""Pins of the FP64 policy reference (oracle/policy.py) against what fixes it independently of
its own code: PyTorch's float64 GRU cell and linear layers (a separate implementation of the
same definitions, App. A: MLP -> GRU -> linear), the gates' saturation limits, a 2-unit step
worked by hand, and the bf16 rounding rule on values whose rounding is known exactly."""
import numpy as np
import pytest

from oracle.policy import bf16_round, policy_actions, policy_step

torch = pytest.importorskip("torch")


def _weights(H, od, seed):
    g = np.random.default_rng(seed)
    return dict(w1=g.normal(0, 0.4, (H, od)), b1=g.normal(0, 0.2, H),
                wi=g.normal(0, 0.3, (3 * H, H)), bi=g.normal(0, 0.2, 3 * H),
                wh=g.normal(0, 0.3, (3 * H, H)), bh=g.normal(0, 0.2, 3 * H),
                wo=g.normal(0, 0.3, (2, H)), bo=g.normal(0, 0.1, 2))


def test_matches_torch_gru_cell_and_linear_layers():
    H, od, rows, vmax = 8, 14, 7, 0.2
    w = _weights(H, od, 1)
    g = np.random.default_rng(2)
    obs, h = g.normal(0, 1, (rows, od)), g.normal(0, 0.5, (rows, H))
    a, hn = policy_step(w, obs, h, vmax)
    cell = torch.nn.GRUCell(H, H).double()
    with torch.no_grad():
        cell.weight_ih.copy_(torch.from_numpy(w["wi"]))
        cell.weight_hh.copy_(torch.from_numpy(w["wh"]))
        cell.bias_ih.copy_(torch.from_numpy(w["bi"]))
        cell.bias_hh.copy_(torch.from_numpy(w["bh"]))
        h1 = torch.relu(torch.nn.functional.linear(torch.from_numpy(obs), torch.from_numpy(w["w1"]),
                                                   torch.from_numpy(w["b1"])))
        ht = cell(h1, torch.from_numpy(h))
        at = vmax * torch.tanh(torch.nn.functional.linear(ht, torch.from_numpy(w["wo"]),
                                                          torch.from_numpy(w["bo"])))
    assert np.abs(hn - ht.numpy()).max() < 1e-13
    assert np.abs(a - at.numpy()).max() < 1e-13


def test_gate_saturation_limits():
    """z -> 1 keeps the state; z -> 0 with r -> 0 makes the new state independent of the old."""
    H, od, rows = 4, 6, 5
    w = _weights(H, od, 3)
    g = np.random.default_rng(4)
    obs, h = g.normal(0, 1, (rows, od)), g.normal(0, 0.5, (rows, H))
    keep = dict(w, bi=w["bi"].copy())
    keep["bi"][H:2 * H] = 60.0  # z = sigma(>= 60 - |.|) = 1 to double precision
    _, hk = policy_step(keep, obs, h, 0.2)
    assert np.abs(hk - h).max() < 1e-20 + 1e-15
    fresh = dict(w, bi=w["bi"].copy())
    fresh["bi"][:H] = -60.0      # r = 0
    fresh["bi"][H:2 * H] = -60.0  # z = 0
    _, h_a = policy_step(fresh, obs, h, 0.2)
    _, h_b = policy_step(fresh, obs, -3.0 * h, 0.2)
    assert np.abs(h_a - h_b).max() < 1e-12


def test_two_unit_step_by_hand():
    """All weights and biases zero except the head: r = z = 1/2 and n = tanh(0) = 0, so the new
    state is h / 2; with Wo = I and bo = 0 the action is v_max (tanh(0.5), tanh(-1))."""
    H, od = 2, 3
    w = dict(w1=np.zeros((H, od)), b1=np.zeros(H), wi=np.zeros((3 * H, H)), bi=np.zeros(3 * H),
             wh=np.zeros((3 * H, H)), bh=np.zeros(3 * H), wo=np.eye(2), bo=np.zeros(2))
    a, hn = policy_step(w, np.array([[0.3, -0.2, 5.0]]), np.array([[1.0, -2.0]]), 0.2)
    assert np.allclose(hn, [[0.5, -1.0]], rtol=0, atol=1e-15)
    # tanh(0.5) = 0.46211715726000974, tanh(1) = 0.76159415595576489 (tables)
    assert np.allclose(a, [[0.2 * 0.46211715726000974, -0.2 * 0.76159415595576489]], atol=1e-15)
    # the ReLU layer: h1 = max(W1 o + b1, 0) enters only through Wi; with Wi_n = I it gives
    # n = tanh(relu(o_0)), tanh(relu(-o_1)) ... checked on one unit: o = (0.7, 0.4, 0)
    w2 = dict(w, w1=np.array([[1.0, 0.0, 0.0], [0.0, -1.0, 0.0]]),
              wi=np.vstack([np.zeros((2 * H, H)), np.eye(H)]))
    _, hn2 = policy_step(w2, np.array([[0.7, 0.4, 0.0]]), np.zeros((1, H)), 0.2)
    # h' = (1 - 1/2) * tanh((0.7, relu(-0.4) = 0)) = (tanh(0.7) / 2, 0); tanh(0.7) = 0.6043677771
    assert np.allclose(hn2, [[0.5 * 0.60436777711716349, 0.0]], atol=1e-15)


def test_bf16_rounding_rule():
    # spacing of bf16 near 1 is 2^-7: 1 + 2^-8 is a tie and goes to the even neighbour 1;
    # 1 + 3 * 2^-8 is a tie between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
    v = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -9, -2.5, 3.0e-3])
    r = bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1 + 2.0 ** -6 and r[3] == 1.0
    assert r[4] == -2.5
    assert abs(r[5] - 3.0e-3) <= 3.0e-3 * 2.0 ** -8  # half an ulp of an 8-bit significand


def test_episode_end_zeroes_the_state():
    """A robot whose env ended at step 0 acts at step 1 as from a zero state."""
    H, od, E, N = 6, 5, 3, 2
    w = _weights(H, od, 5)
    g = np.random.default_rng(6)
    obs_seq = [g.normal(0, 1, (E * N, od)) for _ in range(2)]
    done = [np.array([0, 1, 0], np.uint8), np.zeros(3, np.uint8)]
    row_env = np.repeat(np.arange(E), N)
    acts = policy_actions(w, obs_seq, done, row_env, 0.2)
    fresh, _ = policy_step(w, obs_seq[1], np.zeros((E * N, H)), 0.2)
    assert np.array_equal(acts[1][2:4], fresh[2:4])
    assert not np.allclose(acts[1][:2], fresh[:2])
