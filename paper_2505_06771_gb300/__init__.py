"""Python binding of the GB300 batched multi-robot environment step (include/rl.h).

The environment is JaxRobotarium's (arXiv 2505.06771): GRITSBot unicycles driven through a
single-integrator controller and a barrier-certificate QP safety filter (Sec. 4.1), the
ControllerManager ordering (Sec. 6.1), Navigation and Foraging scenarios (App. B).  Every step
runs in the CUDA library ``_build/librobo_gb300.so``; this module only marshals arguments
(torch tensors -> device pointers, the torch stream -> a cudaStream_t).  There is no CPU path:
if the library is missing the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

from .build import LIB as LIB_PATH
from .build import build

__all__ = ["build", "lib", "config_default", "Env", "Server", "Policy", "RLError", "NAVIGATION",
           "FORAGING", "DISCOVERY", "COUNTERS", "exported_symbols", "rollout_noalloc", "noalloc_state_bytes",
           "noalloc_max_bytes"]

NAVIGATION, FORAGING, DISCOVERY = 0, 1, 2
COUNTERS = ("collisions", "oob", "success", "qp_active", "qp_flagged", "qp_infeasible",
            "episodes", "qp_iters")
_STATUS = {0: "RL_OK", 1: "RL_ERR_ARG", 2: "RL_ERR_CUDA", 3: "RL_ERR_OOM", 4: "RL_ERR_STATE",
           5: "RL_ERR_TIMEOUT", 6: "RL_ERR_BUDGET"}
_HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                    "rl.h")


class RLError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class RLConfig(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("scenario", "precision", "scripted", "episode_len", "n_res_min", "n_res_max",
                 "r_max", "n_max", "max_attempts", "qp_max_iter", "resolve_f64", "lanes",
                 "block_threads", "warp_envs", "small_variant", "controller")] + \
               [(n, ctypes.c_double) for n in
                ("gamma", "r", "l", "vmax", "wmax", "dt", "kappa", "k_si", "noise_amp", "c_col",
                 "forage_radius", "xmin", "xmax", "ymin", "ymax", "init_margin", "min_sep",
                 "near_frac", "near_dmin", "near_dmax", "h_flag", "goal_eps", "pose_k1",
                 "pose_k2", "pose_k3", "sense_radius", "tag_radius", "sense_reward",
                 "tag_reward", "step_penalty")]


class RLRequest(ctypes.Structure):
    _fields_ = [("n_envs", ctypes.c_int32), ("n_robots", ctypes.c_int32),
                ("horizon", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class RLResult(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32), ("n_envs", ctypes.c_int32),
                ("n_robots", ctypes.c_int32), ("horizon", ctypes.c_int32),
                ("submit_s", ctypes.c_double), ("start_s", ctypes.c_double),
                ("finish_s", ctypes.c_double), ("mean_return", ctypes.c_double),
                ("counters", ctypes.c_int32 * 8)]


class RLStepIO(ctypes.Structure):
    _fields_ = [("d_actions", ctypes.c_void_p), ("d_obs", ctypes.c_void_p),
                ("d_reward", ctypes.c_void_p), ("d_done", ctypes.c_void_p),
                ("d_u_nom", ctypes.c_void_p), ("d_u_star", ctypes.c_void_p),
                ("d_vw", ctypes.c_void_p), ("d_qp_info", ctypes.c_void_p)]


_LOCK = threading.Lock()
_LIB = None


def exported_symbols() -> list[str]:
    """Function names declared in include/rl.h."""
    src = open(_HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rl_[a-z_0-9]+)\s*\(", src)))


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library missing ({LIB_PATH}); run "
                               "paper_2505_06771_gb300.build() first")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, u64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64, ctypes.c_size_t
        L.rl_config_default.argtypes = [i32, ctypes.POINTER(RLConfig)]
        L.rl_create.argtypes = [ctypes.POINTER(RLConfig), i32, vp, i32, u64, vp,
                                ctypes.POINTER(vp)]
        L.rl_reset.argtypes = [vp, u64]
        L.rl_step.argtypes = [vp, vp, vp, vp, vp]
        L.rl_step_io_call.argtypes = [vp, ctypes.POINTER(RLStepIO)]
        L.rl_rollout.argtypes = [vp, i32, vp, vp, vp]
        L.rl_rollout_plain.argtypes = [vp, i32, vp, vp, vp]
        L.rl_rollout_host.argtypes = [vp, vp, i32, vp, vp, vp]
        L.rl_state_bytes.argtypes = [vp]
        L.rl_state_bytes.restype = sz
        L.rl_get_state.argtypes = [vp, vp, sz]
        L.rl_set_state.argtypes = [vp, vp, sz]
        L.rl_get_counters.argtypes = [vp, vp]
        L.rl_sync.argtypes = [vp]
        for f in ("rl_obs_dim", "rl_n_envs", "rl_total_robots", "rl_lanes"):
            getattr(L, f).argtypes = [vp]
            getattr(L, f).restype = i32
        L.rl_last_error.argtypes = [vp]
        L.rl_last_error.restype = ctypes.c_char_p
        L.rl_destroy.argtypes = [vp]
        L.rl_destroy.restype = None
        L.rl_tune.argtypes = [vp, i32, vp]
        L.rl_set_class_launch.argtypes = [vp, i32]
        L.rl_server_create.argtypes = [ctypes.POINTER(RLConfig), sz, i32, ctypes.POINTER(vp)]
        L.rl_server_submit.argtypes = [vp, ctypes.POINTER(RLRequest),
                                       ctypes.POINTER(ctypes.c_uint64)]
        L.rl_server_result.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(RLResult), vp]
        L.rl_server_stats.argtypes = [vp, vp]
        L.rl_server_drain.argtypes = [vp, ctypes.c_double]
        L.rl_server_destroy.argtypes = [vp]
        L.rl_rollout_noalloc.argtypes = [ctypes.POINTER(RLConfig), i32, i32, u64, i32, vp, vp, vp,
                                         vp]
        L.rl_noalloc_state_bytes.argtypes = [ctypes.POINTER(RLConfig), i32, i32]
        L.rl_noalloc_state_bytes.restype = sz
        L.rl_policy_create.argtypes = [vp, i32] + [vp] * 8 + [ctypes.POINTER(vp)]
        L.rl_policy_reset_hidden.argtypes = [vp]
        L.rl_policy_rollout.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp]
        L.rl_policy_destroy.argtypes = [vp]
        L.rl_policy_destroy.restype = None
        L.rl_observe.argtypes = [vp, vp]
        _LIB = L
        return L


def config_default(scenario: int = NAVIGATION, **overrides) -> dict:
    c = RLConfig()
    st = lib().rl_config_default(scenario, ctypes.byref(c))
    if st:
        raise RLError(st, "rl_config_default")
    d = {name: getattr(c, name) for name, _ in RLConfig._fields_}
    for k in overrides:
        if k not in d:
            raise KeyError(k)
    d.update(overrides)
    return d


def _to_struct(cfg: dict) -> RLConfig:
    c = RLConfig()
    for name, _ in RLConfig._fields_:
        setattr(c, name, cfg[name])
    return c


def _dptr(t, dtype, numel=None, name="buffer"):
    """Device pointer of a contiguous CUDA tensor of the expected dtype (or None)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name}: expected a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name}: needs {numel} elements, has {t.numel()}")
    return t.data_ptr()


def _hptr(a, numel, itemsize, name):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"] or a.nbytes < numel * itemsize:
            raise ValueError(f"{name}: contiguous host array of {numel} items needed")
        return a.ctypes.data
    import torch
    if isinstance(a, torch.Tensor) and not a.is_cuda and a.is_contiguous():
        if a.numel() * a.element_size() < numel * itemsize:
            raise ValueError(f"{name}: too small")
        return a.data_ptr()
    raise TypeError(f"{name}: expected a contiguous host array")


class Env:
    """A batch of environments on the current CUDA device (one rl_env handle)."""

    def __init__(self, cfg: dict, n_envs: int, n_robots, seed: int = 0, stream=None):
        import torch
        L = lib()
        self._L = L
        self.cfg = dict(cfg)
        if isinstance(n_robots, (int, np.integer)):
            arr, uni = None, int(n_robots)
            self.n_robots = np.full(n_envs, uni, np.int32)
        else:
            arr = np.ascontiguousarray(n_robots, dtype=np.int32)
            if len(arr) != n_envs:
                raise ValueError("n_robots must have n_envs entries")
            uni = 0
            self.n_robots = arr
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        st = L.rl_create(ctypes.byref(_to_struct(self.cfg)), n_envs,
                         None if arr is None else arr.ctypes.data, uni, seed,
                         ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if st:
            raise RLError(st, "rl_create")
        self._h = h
        self.n_envs = n_envs
        self.obs_dim = int(L.rl_obs_dim(h))
        self.total_robots = int(L.rl_total_robots(h))
        self.lanes = int(L.rl_lanes(h))
        self.dtype = torch.float64 if self.cfg["precision"] == 64 else torch.float32
        self.np_dtype = np.float64 if self.cfg["precision"] == 64 else np.float32
        self.off = np.concatenate([[0], np.cumsum(self.n_robots)]).astype(np.int64)

    # ------------------------------------------------------------------ calls
    def _check(self, st, what):
        if st:
            raise RLError(st, f"{what}: {self._L.rl_last_error(self._h).decode()}")

    def reset(self, seed: int):
        self._check(self._L.rl_reset(self._h, seed), "rl_reset")

    def step(self, actions=None, obs=None, reward=None, done=None, u_nom=None, u_star=None,
             vw=None, qp_info=None):
        import torch
        R, E = self.total_robots, self.n_envs
        io = RLStepIO(_dptr(actions, self.dtype, 2 * R, "actions"),
                      _dptr(obs, self.dtype, R * self.obs_dim, "obs"),
                      _dptr(reward, self.dtype, E, "reward"),
                      _dptr(done, torch.uint8, E, "done"),
                      _dptr(u_nom, self.dtype, 2 * R, "u_nom"),
                      _dptr(u_star, self.dtype, 2 * R, "u_star"),
                      _dptr(vw, self.dtype, 2 * R, "vw"),
                      _dptr(qp_info, torch.int32, 4 * E, "qp_info"))
        self._check(self._L.rl_step_io_call(self._h, ctypes.byref(io)), "rl_step")

    def rollout(self, T: int, obs=None, reward=None, done=None, plain: bool = False):
        import torch
        R, E = self.total_robots, self.n_envs
        f = self._L.rl_rollout_plain if plain else self._L.rl_rollout
        self._check(f(self._h, T, _dptr(obs, self.dtype, T * R * self.obs_dim, "obs"),
                      _dptr(reward, self.dtype, T * E, "reward"),
                      _dptr(done, torch.uint8, T * E, "done")), "rl_rollout")

    def rollout_host(self, T: int, state=None, obs=None, reward=None, done=None):
        R, E = self.total_robots, self.n_envs
        isz = 8 if self.cfg["precision"] == 64 else 4
        sp = None
        if state is not None:
            sb = np.frombuffer(state, np.uint8) if isinstance(state, (bytes, bytearray)) else state
            sp = _hptr(sb, self.state_bytes(), 1, "state")
        self._check(self._L.rl_rollout_host(self._h, sp, T,
                                            _hptr(obs, T * R * self.obs_dim, isz, "obs"),
                                            _hptr(reward, T * E, isz, "reward"),
                                            _hptr(done, T * E, 1, "done")), "rl_rollout_host")

    def tune(self, T_probe: int = 50) -> dict:
        """rl_tune: pick the fastest launch shape for this batch; returns the choice."""
        out = np.zeros(26, np.int32)
        self._check(self._L.rl_tune(self._h, T_probe, out.ctypes.data), "rl_tune")
        self.lanes = int(self._L.rl_lanes(self._h))
        return {"one_launch": bool(out[0] == 1), "class_launch": int(out[0]),
                "classes": [dict(nmax=int(out[1 + 5 * c]), lanes=int(out[2 + 5 * c]),
                                 block_threads=int(out[3 + 5 * c]),
                                 warp_envs=int(out[4 + 5 * c]), variant=int(out[5 + 5 * c]))
                            for c in range(5) if out[1 + 5 * c] > 0]}

    def set_class_launch(self, mode: int):
        """rl_set_class_launch: uneven batches as one persistent launch (1), one launch per class
        in sequence (0) or one per class on parallel streams (2)."""
        self._check(self._L.rl_set_class_launch(self._h, int(mode)), "rl_set_class_launch")

    def state_bytes(self) -> int:
        return int(self._L.rl_state_bytes(self._h))

    def get_state(self) -> bytes:
        n = self.state_bytes()
        buf = ctypes.create_string_buffer(n)
        self._check(self._L.rl_get_state(self._h, buf, n), "rl_get_state")
        return buf.raw

    def set_state(self, blob: bytes):
        self._check(self._L.rl_set_state(self._h, blob, len(blob)), "rl_set_state")

    def counters(self) -> np.ndarray:
        out = np.zeros((self.n_envs, 8), np.int32)
        self._check(self._L.rl_get_counters(self._h, out.ctypes.data), "rl_get_counters")
        return out

    def sync(self):
        self._check(self._L.rl_sync(self._h), "rl_sync")

    def observe(self, obs):
        """rl_observe: the observation of the current state into obs [rows, obs_dim]."""
        self._check(self._L.rl_observe(self._h, _dptr(obs, self.dtype,
                                                       self.total_robots * self.obs_dim, "obs")),
                    "rl_observe")

    def close(self):
        if getattr(self, "_h", None):
            self._L.rl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ state blob
    def state_arrays(self, blob: bytes | None = None) -> dict:
        """Parse a state blob (header + image of 256-byte-aligned segments) into arrays."""
        return parse_state(blob if blob is not None else self.get_state())


class Policy:
    """rl_policy_*: an MLP (ReLU) -> GRU -> linear policy evaluated on the GPU between steps of
    a policy-driven binary32 handle.  weights: dict of float32 arrays w1 [H, obs_dim], b1 [H],
    wi [3H, H], bi [3H], wh [3H, H], bh [3H] (gates r, z, n), wo [2, H], bo [2]."""

    NAMES = ("w1", "b1", "wi", "bi", "wh", "bh", "wo", "bo")

    def __init__(self, env: "Env", weights: dict):
        self._L = lib()
        self.env = env
        H = int(np.asarray(weights["b1"]).shape[0])
        self.hidden = H
        self._w = [np.ascontiguousarray(weights[k], dtype=np.float32) for k in self.NAMES]
        h = ctypes.c_void_p()
        st = self._L.rl_policy_create(env._h, H, *[a.ctypes.data for a in self._w],
                                      ctypes.byref(h))
        if st != 0:
            raise RLError(st, "rl_policy_create: " + self._L.rl_last_error(env._h).decode())
        self._h = h

    def reset_hidden(self):
        st = self._L.rl_policy_reset_hidden(self._h)
        if st != 0:
            raise RLError(st, "rl_policy_reset_hidden")

    def rollout(self, T: int, obs0, obs, done, reward=None, actions=None):
        """T policy-driven steps: obs0 [rows, od] -> obs [T, rows, od], done [T, E], reward
        [T, E] and actions [T, rows, 2] (optional)."""
        import torch
        e = self.env
        R, E, od = e.total_robots, e.n_envs, e.obs_dim
        st = self._L.rl_policy_rollout(
            e._h, self._h, T, _dptr(obs0, torch.float32, R * od, "obs0"),
            _dptr(obs, torch.float32, T * R * od, "obs"),
            _dptr(reward, torch.float32, T * E, "reward"),
            _dptr(done, torch.uint8, T * E, "done"),
            _dptr(actions, torch.float32, T * R * 2, "actions"))
        if st != 0:
            raise RLError(st, "rl_policy_rollout: " + self._L.rl_last_error(e._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.rl_policy_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rollout_noalloc(cfg: dict, n_envs: int, n_robots: int, seed: int, T: int, obs=None,
                    reward=None, done=None, stream=None):
    """rl_rollout_noalloc: reset + T scripted steps with the state in the library's static
    device array (no allocation).  Buffers as for Env.rollout; stream: a torch stream or None
    for the current one."""
    import torch
    L = lib()
    dt = torch.float64 if cfg["precision"] == 64 else torch.float32
    rows = n_envs * n_robots
    n_max = cfg["n_max"] if cfg["n_max"] > 0 else n_robots
    od = {FORAGING: 4 + 4 * (n_max - 1) + 4 * cfg["r_max"],
          DISCOVERY: 5 + 5 * (n_max - 1) + 4 * cfg["r_max"]}.get(cfg["scenario"],
                                                                 5 + 3 * (n_max - 1))
    s = stream if stream is not None else torch.cuda.current_stream()
    st = L.rl_rollout_noalloc(ctypes.byref(_to_struct(cfg)), n_envs, n_robots, seed, T,
                              _dptr(obs, dt, T * rows * od, "obs"),
                              _dptr(reward, dt, T * n_envs, "reward"),
                              _dptr(done, torch.uint8, T * n_envs, "done"),
                              ctypes.c_void_p(s.cuda_stream))
    if st:
        raise RLError(st, "rl_rollout_noalloc")


class Server:
    """Continuous-batching rollout server (rl_server_*) on the current CUDA device."""

    def __init__(self, cfg: dict, hbm_budget_bytes: int, max_slots: int = 16):
        import torch
        torch.cuda.current_device()
        self._L = lib()
        h = ctypes.c_void_p()
        st = self._L.rl_server_create(ctypes.byref(_to_struct(cfg)), int(hbm_budget_bytes),
                                      max_slots, ctypes.byref(h))
        if st:
            raise RLError(st, "rl_server_create")
        self._h = h

    def submit(self, n_envs: int, n_robots: int, horizon: int, seed: int) -> int:
        rid = ctypes.c_uint64()
        st = self._L.rl_server_submit(self._h, ctypes.byref(RLRequest(n_envs, n_robots, horizon,
                                                                      seed)), ctypes.byref(rid))
        if st:
            raise RLError(st, "rl_server_submit")
        return int(rid.value)

    def result(self, rid: int, returns: bool = False):
        r = RLResult()
        buf = None
        st = self._L.rl_server_result(self._h, rid, ctypes.byref(r), None)
        if st == 0 and returns and r.status == 2:
            buf = np.zeros(r.n_envs, np.float32)
            st = self._L.rl_server_result(self._h, rid, ctypes.byref(r), buf.ctypes.data)
        if st:
            raise RLError(st, "rl_server_result")
        d = {k: getattr(r, k) for k, _ in RLResult._fields_ if k != "counters"}
        d["counters"] = list(r.counters)
        d["latency_s"] = r.finish_s - r.submit_s
        if buf is not None:
            d["returns"] = buf
        return d

    def stats(self) -> dict:
        out = np.zeros(6, np.int64)
        self._L.rl_server_stats(self._h, out.ctypes.data)
        return dict(used=int(out[0]), peak=int(out[1]), done=int(out[2]), running=int(out[3]),
                    queued=int(out[4]), env_steps=int(out[5]))

    def drain(self, timeout_s: float) -> bool:
        st = self._L.rl_server_drain(self._h, timeout_s)
        if st not in (0, 5):
            raise RLError(st, "rl_server_drain")
        return st == 0

    def close(self):
        if getattr(self, "_h", None):
            self._L.rl_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def noalloc_state_bytes(cfg: dict, n_envs: int, n_robots: int) -> int:
    return int(lib().rl_noalloc_state_bytes(ctypes.byref(_to_struct(cfg)), n_envs, n_robots))


def noalloc_max_bytes() -> int:
    """RL_NOALLOC_MAX_BYTES as include/rl.h defines it: the state a no-allocation rollout holds."""
    m = re.search(r"#define\s+RL_NOALLOC_MAX_BYTES\s+\(\(size_t\)(\d+)\s*<<\s*(\d+)\)",
                  open(_HDR).read())
    if not m:
        raise RuntimeError("RL_NOALLOC_MAX_BYTES not found in include/rl.h")
    return int(m.group(1)) << int(m.group(2))


_SEGS = [("x", "r", "T"), ("y", "r", "T"), ("th", "r", "T"), ("gx", "r", "T"), ("gy", "r", "T"),
         ("level", "i", "T"), ("t", "i", "E"), ("ep", "i", "E"), ("n_res", "i", "E"),
         ("qx", "r", "RM"), ("qy", "r", "RM"), ("qlevel", "i", "RM"), ("qactive", "i", "RM"),
         ("counters", "i", "C"), ("n_robots", "i", "E"), ("off", "i", "E1"), ("gth", "r", "T")]


def parse_state(blob: bytes) -> dict:
    hdr = np.frombuffer(blob, np.int32, 10)
    magic, version, prec, scen, E, T, rmax, nmax = [int(v) for v in hdr[:8]]
    if magic != 0x31534C52 or version != 2:
        raise ValueError("not a state blob")
    seed, img = np.frombuffer(blob, np.uint64, 2, offset=32)
    rdt = np.float64 if prec == 64 else np.float32
    counts = dict(T=T, E=E, RM=E * rmax, C=E * 8, E1=E + 1)
    out = dict(precision=prec, scenario=scen, n_envs=E, total_robots=T, r_max=rmax, n_max=nmax,
               seed=int(seed))
    pos = 64
    for name, kind, cnt in _SEGS:
        dt = rdt if kind == "r" else np.int32
        n = counts[cnt]
        nbytes = n * np.dtype(dt).itemsize
        out[name] = np.frombuffer(blob, dt, n, offset=pos).copy()
        pos += (nbytes + 255) & ~255
    out["counters"] = out["counters"].reshape(E, 8)
    return out
