"""FP64 CPU oracle of the batched multi-robot environment step (JaxRobotarium, arXiv 2505.06771).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import this package.  It shares no code with the CUDA library in
``paper_2505_06771_gb300/`` and never imports it.

The arithmetic lives in ``oracle.c`` (plain C, double precision); this module only compiles it
with gcc and marshals numpy arrays through ctypes.  Paper passages followed: Sec. 4.1 (unicycle
model, single-integrator controller, barrier-certificate QP), Sec. 6.1 (controller -> barrier ->
robot ordering), Sec. 7 (action noise), App. B (Navigation and Foraging observations, rewards,
episode length).

Parity status: every function here is pinned by ``tests/test_oracle_*.py`` (Philox known-answer
vectors, closed-form Euler arcs, brute-force QP enumeration, KKT residuals, the half-plane
projection, forward invariance, subset enumeration for the foraging rule).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_LOCK = threading.Lock()
_LIB = None

NAV, FORAGE, DISCOVERY = 0, 1, 2
NCOUNT = 8
CNT_COLLISIONS, CNT_OOB, CNT_SUCCESS, CNT_QP_ACTIVE = 0, 1, 2, 3
CNT_QP_FLAGGED, CNT_QP_INFEASIBLE, CNT_EPISODES, CNT_QP_ITERS = 4, 5, 6, 7


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, -O2, OpenMP, no FP contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(src), os.path.getmtime(hdr))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-D_DEFAULT_SOURCE", src, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class Cfg(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("scenario", "scripted", "episode_len", "n_res_min", "n_res_max", "max_attempts",
                 "n_max", "r_max", "controller")] + \
               [(n, ctypes.c_double) for n in
                ("gamma", "r", "l", "vmax", "wmax", "dt", "kappa", "k_si", "noise_amp", "c_col",
                 "forage_radius", "xmin", "xmax", "ymin", "ymax", "init_margin", "min_sep",
                 "near_frac", "near_dmin", "near_dmax", "goal_eps", "pose_k1", "pose_k2",
                 "pose_k3", "sense_radius", "tag_radius", "sense_reward", "tag_reward",
                 "step_penalty")]


_P = ctypes.POINTER
_D, _I, _U8 = ctypes.c_double, ctypes.c_int32, ctypes.c_uint8


class _Batch(ctypes.Structure):
    _fields_ = [("x", _P(_D)), ("y", _P(_D)), ("th", _P(_D)), ("gx", _P(_D)), ("gy", _P(_D)),
                ("gth", _P(_D)), ("level", _P(_I)), ("t", _P(_I)), ("ep", _P(_I)), ("n_res", _P(_I)),
                ("qx", _P(_D)), ("qy", _P(_D)), ("qlevel", _P(_I)), ("qactive", _P(_I)),
                ("counters", _P(_I))]


class _Trace(ctypes.Structure):
    _fields_ = [("u_nom", _P(_D)), ("u_star", _P(_D)), ("vw", _P(_D)), ("qp", _P(_I)),
                ("kkt", _P(_D))]


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            lib.orc_philox4x32_10.argtypes = [_P(ctypes.c_uint32), _P(ctypes.c_uint32),
                                              _P(ctypes.c_uint32)]
            lib.orc_obs_dim.argtypes = [_P(Cfg)]
            lib.orc_reset_batch.argtypes = [_P(Cfg), ctypes.c_uint64, ctypes.c_int, _P(_I), _P(_I),
                                            _P(_Batch)]
            lib.orc_step_batch.argtypes = [_P(Cfg), ctypes.c_uint64, ctypes.c_int, _P(_I),
                                           _P(_Batch), _P(_D), _P(_D), _P(_D), _P(_U8),
                                           _P(_Trace), ctypes.c_int]
            lib.orc_rollout.argtypes = [_P(Cfg), ctypes.c_uint64, ctypes.c_int, _P(_I),
                                        _P(_Batch), ctypes.c_int, _P(_D), _P(_D), _P(_U8),
                                        ctypes.c_int]
            lib.orc_qp_project.argtypes = [ctypes.c_int, ctypes.c_int, _P(_D), _P(_D), _P(_D),
                                           _P(_D), _P(_D), _P(_I), _P(_I)]
            lib.orc_build_cbf_rows.argtypes = [_P(Cfg), ctypes.c_int, _P(_D), _P(_D), _P(_D),
                                               _P(_D)]
            lib.orc_unicycle_update.argtypes = [_P(Cfg), _D, _D, _P(_D), _P(_D)]
            lib.orc_unicycle_update.restype = None
            lib.orc_philox4x32_10.restype = None
            _LIB = lib
    return _LIB


def default_cfg(scenario: int = NAV, n_max: int = 4, **overrides) -> dict:
    """Constants of the step.  Barrier gain 100, safety radius 0.17 m, projection distance
    0.05 m, |v| <= 0.2 m/s, |omega| <= 3.6 rad/s, dt = 0.033 s, arena 3.2 x 2.0 m centred at
    the origin, 100-step episodes (App. B), boundary gain factor 0.4, SI gain 1.0, noise
    U(-0.05, 0.05), collision penalty 1 (Navigation) / 0 (Foraging, App. B), foraging radius
    0.25 m, initial poses >= 0.3 m apart and >= 0.2 m from the walls."""
    c = dict(scenario=scenario, scripted=1, episode_len=100, n_res_min=2, n_res_max=6,
             max_attempts=4096, n_max=n_max, r_max=0 if scenario == NAV else 6,
             gamma=100.0, r=0.17, l=0.05, vmax=0.2, wmax=3.6, dt=0.033, kappa=0.4, k_si=1.0,
             noise_amp=0.05, c_col=1.0 if scenario == NAV else 0.0, forage_radius=0.25,
             sense_radius=0.45, tag_radius=0.25, sense_reward=1.0, tag_reward=5.0,
             step_penalty=0.05,
             xmin=-1.6, xmax=1.6, ymin=-1.0, ymax=1.0, init_margin=0.2, min_sep=0.3,
             near_frac=0.0, near_dmin=0.18, near_dmax=0.20, goal_eps=0.0, controller=0,
             pose_k1=1.0, pose_k2=2.0, pose_k3=1.0)
    c.update(overrides)
    return c


def _cfg(c: dict) -> Cfg:
    s = Cfg()
    for name, _ in Cfg._fields_:
        setattr(s, name, c[name])
    return s


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(_P(ctype))


def obs_dim(c: dict) -> int:
    return int(_lib().orc_obs_dim(ctypes.byref(_cfg(c))))


class State:
    """Batched SoA state in double precision (robots of env e at rows off[e] .. off[e]+n[e])."""

    def __init__(self, c: dict, n_robots):
        self.n_robots = np.ascontiguousarray(n_robots, dtype=np.int32)
        E = len(self.n_robots)
        tot = int(self.n_robots.sum())
        R = max(int(c["r_max"]), 1)
        self.r_max = int(c["r_max"])
        self.off = np.concatenate([[0], np.cumsum(self.n_robots)]).astype(np.int64)
        for name in ("x", "y", "th", "gx", "gy", "gth"):
            setattr(self, name, np.zeros(tot, np.float64))
        self.level = np.zeros(tot, np.int32)
        self.t = np.zeros(E, np.int32)
        self.ep = np.zeros(E, np.int32)
        self.n_res = np.zeros(E, np.int32)
        self.qx = np.zeros(E * R, np.float64)
        self.qy = np.zeros(E * R, np.float64)
        self.qlevel = np.zeros(E * R, np.int32)
        self.qactive = np.zeros(E * R, np.int32)
        self.counters = np.zeros(E * NCOUNT, np.int32)

    def copy(self) -> "State":
        s = State.__new__(State)
        for k, v in self.__dict__.items():
            setattr(s, k, v.copy() if isinstance(v, np.ndarray) else v)
        return s

    def _c(self) -> _Batch:
        b = _Batch()
        for name in ("x", "y", "th", "gx", "gy", "gth", "qx", "qy"):
            setattr(b, name, _ptr(getattr(self, name), _D))
        for name in ("level", "t", "ep", "n_res", "qlevel", "qactive", "counters"):
            setattr(b, name, _ptr(getattr(self, name), _I))
        return b


def reset(c: dict, seed: int, n_robots, ep=None) -> State:
    s = State(c, n_robots)
    epa = None if ep is None else np.ascontiguousarray(ep, dtype=np.int32)
    b = s._c()
    rc = _lib().orc_reset_batch(ctypes.byref(_cfg(c)), seed, len(s.n_robots),
                                _ptr(s.n_robots, _I), _ptr(epa, _I), ctypes.byref(b))
    if rc:
        raise ValueError(f"orc_reset_batch failed ({rc})")
    return s


def step(c: dict, seed: int, s: State, actions=None, trace: bool = False, threads: int = 0):
    """One step of every env (in place on ``s``).  Returns obs [sum n, obs_dim], reward [E],
    done [E] and, with ``trace``, a dict of u_nom, u_star, vw, qp [E,4], kkt [E]."""
    E = len(s.n_robots)
    tot = int(s.off[-1])
    od = obs_dim(c)
    obs = np.zeros((tot, od), np.float64)
    rew = np.zeros(E, np.float64)
    done = np.zeros(E, np.uint8)
    act = None if actions is None else np.ascontiguousarray(actions, dtype=np.float64).reshape(-1)
    tr = None
    trd = None
    if trace:
        trd = dict(u_nom=np.zeros((tot, 2)), u_star=np.zeros((tot, 2)), vw=np.zeros((tot, 2)),
                   qp=np.zeros((E, 4), np.int32), kkt=np.zeros(E))
        tr = _Trace(_ptr(trd["u_nom"], _D), _ptr(trd["u_star"], _D), _ptr(trd["vw"], _D),
                    _ptr(trd["qp"], _I), _ptr(trd["kkt"], _D))
    b = s._c()
    rc = _lib().orc_step_batch(ctypes.byref(_cfg(c)), seed, E, _ptr(s.n_robots, _I),
                               ctypes.byref(b), _ptr(act, _D), _ptr(obs, _D), _ptr(rew, _D),
                               _ptr(done, _U8), ctypes.byref(tr) if tr is not None else None,
                               threads)
    if rc:
        raise ValueError(f"orc_step_batch failed ({rc})")
    return obs, rew, done, trd


def rollout(c: dict, seed: int, s: State, T: int, want_obs: bool = True, threads: int = 0):
    """T scripted steps of every env (in place on ``s``): obs [T, sum n, obs_dim] (or None),
    reward [T, E], done [T, E]."""
    E = len(s.n_robots)
    tot = int(s.off[-1])
    od = obs_dim(c)
    obs = np.zeros((T, tot, od), np.float64) if want_obs else None
    rew = np.zeros((T, E), np.float64)
    done = np.zeros((T, E), np.uint8)
    b = s._c()
    rc = _lib().orc_rollout(ctypes.byref(_cfg(c)), seed, E, _ptr(s.n_robots, _I),
                            ctypes.byref(b), T, _ptr(obs, _D), _ptr(rew, _D), _ptr(done, _U8),
                            threads)
    if rc:
        raise ValueError(f"orc_rollout failed ({rc})")
    return obs, rew, done


def qp_project(A, b, u0):
    """min 1/2 |u - u0|^2 s.t. A u <= b.  Returns (u, lam, status, n_active, iters)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    m, n = A.shape
    u = np.zeros(n)
    lam = np.zeros(m)
    q = _I(0)
    it = _I(0)
    st = _lib().orc_qp_project(n, m, _ptr(A, _D), _ptr(b, _D), _ptr(u0, _D), _ptr(u, _D),
                               _ptr(lam, _D), ctypes.byref(q), ctypes.byref(it))
    return u, lam, int(st), int(q.value), int(it.value)


def pose_control(c: dict, pose, goal):
    """Nominal unicycle command (v, omega) of the pose controller from pose and goal [x, y, th]."""
    p = np.ascontiguousarray(pose, dtype=np.float64)
    g = np.ascontiguousarray(goal, dtype=np.float64)
    vw = np.zeros(2)
    _lib().orc_pose_control(ctypes.byref(_cfg(c)), _ptr(p, _D), _ptr(g, _D), _ptr(vw, _D))
    return vw


def cbf_rows(c: dict, px, py):
    """Barrier QP rows (A [m, 2N], b [m]) of one env from its projected points."""
    px = np.ascontiguousarray(px, dtype=np.float64)
    py = np.ascontiguousarray(py, dtype=np.float64)
    N = len(px)
    m = N * (N - 1) // 2 + 4 * N
    A = np.zeros((m, 2 * N))
    b = np.zeros(m)
    _lib().orc_build_cbf_rows(ctypes.byref(_cfg(c)), N, _ptr(px, _D), _ptr(py, _D), _ptr(A, _D),
                              _ptr(b, _D))
    return A, b


def unicycle_update(c: dict, ux: float, uy: float, pose):
    """SI velocity -> unicycle command -> wheel clip -> one Euler step.  Returns (pose', (v, w))."""
    p = np.ascontiguousarray(pose, dtype=np.float64).copy()
    vw = np.zeros(2)
    _lib().orc_unicycle_update(ctypes.byref(_cfg(c)), float(ux), float(uy), _ptr(p, _D),
                               _ptr(vw, _D))
    return p, vw


def philox4x32_10(ctr, key):
    """Philox4x32-10 block: four 32-bit counter words, two key words -> four output words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, np.uint32)
    _lib().orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                             _ptr(o, ctypes.c_uint32))
    return o
