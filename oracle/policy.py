"""FP64 reference of the recurrent policy evaluated between environment steps.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/`` and the CPU-oracle leg
of ``bench.py`` may import it; it shares no code with the CUDA library.

The policy has the shape the paper trains with (App. A, policy architecture: one dense layer
with ReLU, a GRU, one dense layer; widths 128-512).  For one robot with observation o and
recurrent state h:

    h1 = ReLU(W1 o + b1)
    r  = sigma(Wi_r h1 + bi_r + Wh_r h + bh_r)
    z  = sigma(Wi_z h1 + bi_z + Wh_z h + bh_z)
    n  = tanh(Wi_n h1 + bi_n + r * (Wh_n h + bh_n))
    h' = (1 - z) * n + z * h
    a  = v_max * tanh(Wo h' + bo)

with the gate blocks of Wi, Wh, bi, bh in the order r, z, n.  The state of a robot is zeroed
before the step that follows its env's episode end.  The action a is the robot's nominal
single-integrator velocity for the next environment step.

``bf16=True`` rounds the operands of the two dense products that precede the gates to bf16
(nearest, ties to even) as the GPU's tensor-core path does: o, W1, b1, h1, Wi, Wh and the
previous state fed to the product; accumulation, gates, state and head stay in float64 here.
Parity status: pinned by ``tests/test_oracle_policy.py`` (PyTorch's GRU cell and linear layers
in float64 as independent implementations, gate saturation limits, a hand-computed 2-unit
step).
"""
from __future__ import annotations

import numpy as np


def bf16_round(a):
    """Round to bf16 (nearest, ties to even) and widen back to float64."""
    b = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _sigma(v):
    return 1.0 / (1.0 + np.exp(-v))


def policy_step(w: dict, obs, h, vmax: float, bf16: bool = False):
    """One policy evaluation for every row: obs [rows, od], h [rows, H] -> (action [rows, 2],
    new state [rows, H])."""
    H = np.asarray(w["b1"]).shape[0]
    f = bf16_round if bf16 else (lambda a: np.asarray(a, np.float64))
    W1, b1 = f(w["w1"]), f(w["b1"])
    Wi, Wh = f(w["wi"]), f(w["wh"])
    bi, bh = np.asarray(w["bi"], np.float64), np.asarray(w["bh"], np.float64)
    Wo, bo = np.asarray(w["wo"], np.float64), np.asarray(w["bo"], np.float64)
    h = np.asarray(h, np.float64)
    h1 = np.maximum(f(obs) @ W1.T + b1, 0.0)
    gi = f(h1) @ Wi.T + bi
    gh = f(h) @ Wh.T + bh
    r = _sigma(gi[:, :H] + gh[:, :H])
    z = _sigma(gi[:, H:2 * H] + gh[:, H:2 * H])
    n = np.tanh(gi[:, 2 * H:] + r * gh[:, 2 * H:])
    hn = (1.0 - z) * n + z * h
    return vmax * np.tanh(hn @ Wo.T + bo), hn


def policy_actions(w: dict, obs_seq, done_seq, row_env, vmax: float, bf16: bool = False):
    """Actions of T consecutive steps: obs_seq[t] [rows, od] is the observation feeding step t,
    done_seq[t] [E] the done flags of step t (a robot's state is zeroed before step t + 1 when
    its env ended at step t); the state starts at zero.  Returns [T, rows, 2]."""
    rows = np.asarray(obs_seq[0]).shape[0]
    H = np.asarray(w["b1"]).shape[0]
    h = np.zeros((rows, H))
    acts = []
    for t, o in enumerate(obs_seq):
        if t > 0:
            h[np.asarray(done_seq[t - 1])[row_env].astype(bool)] = 0.0
        a, h = policy_step(w, o, h, vmax, bf16)
        acts.append(a)
    return np.stack(acts)
