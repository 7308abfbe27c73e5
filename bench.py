#!/usr/bin/env python
"""Benchmark of the batched CBF-QP multi-robot environment step on GB300.

Default workload (one bench step): the Navigation batch of 4096 environments x 4 robots,
1000 scripted steps (10 episodes of 100 steps), binary32, run by rl_rollout as one CUDA-graph
replay of the persistent kernel, streaming observations [1000, 16384, 14], rewards and done
flags (938 MB) to HBM.  Reported: env-steps/s (and robot-steps/s), the plain one-launch-per-env-
per-step form of the same step, p50/p99 rollout latency, the HBM roofline fraction of the
rollout kernel, the end-to-end rate through host buffers, and the FP64 CPU oracle timed on the
host cores.

Other workloads (--workload): tiny (16 x 4 x 100, binary64), uneven (8192 envs of 2..10 robots,
Foraging, 500 steps, one persistent launch), largen (1024 x 20 x 300, 30% near pairs, binary32
with binary64 re-solve), serving (Poisson arrivals, 60 GB budget, p50/p99 latency), sweep
(env-steps/s of the Navigation rollout over the number of environments, the GPU analogue of the
paper's parallel-scaling experiment, Sec. 4.2 and Fig. 2).

python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--workload NAME]
Under torchrun each rank runs its own batch (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "env-steps/s with CBF-QP filter vs plain per-env form; p50/p99 rollout latency"

WORKLOADS = {
    "nav": dict(desc="navigation: 4096 envs x 4 robots x 1000 steps, scripted nominal control, fp32",
                scenario=0, E=4096, N=4, T=1000, precision=32, near=0.0, n_max=4),
    "tiny": dict(desc="navigation: 16 envs x 4 robots x 100 steps, fp64",
                 scenario=0, E=16, N=4, T=100, precision=64, near=0.0, n_max=4),
    "uneven": dict(desc="foraging: 8192 envs x U{2..10} robots x 500 steps, 2-6 resources, fp32, "
                        "one persistent launch",
                   scenario=1, E=8192, N="uneven", T=500, precision=32, near=0.0, n_max=10),
    "largen": dict(desc="navigation: 1024 envs x 20 robots x 300 steps, 30% near pairs, fp32 + "
                        "fp64 re-solve of flagged QPs",
                   scenario=0, E=1024, N=20, T=300, precision=32, near=0.3, n_max=20),
    "waypoint": dict(desc="random waypoint navigation: 1 env x 4 robots x 10000 steps, a new goal "
                          "on arrival within 0.05 m, fp32 (the single-env latency workload of "
                          "the paper's Sec. 4.2, Table 2)",
                     scenario=0, E=1, N=4, T=10000, precision=32, near=0.0, n_max=4,
                     goal_eps=0.05, episode_len=10000,
                     context={"paper_table2_ms_per_10k_steps": 9.18,
                              "paper_hardware": "JAX on an Apple M4 Pro CPU (position "
                                                "controller); another machine: context only"}),
    "discovery": dict(desc="discovery: 4096 envs x 4 robots (2 sensing, 2 tagging) x 1000 steps, "
                           "U{2..6} landmarks, fp32",
                      scenario=2, E=4096, N=4, T=1000, precision=32, near=0.0, n_max=4),
    "waypoint_pose": dict(desc="random waypoint navigation under the unicycle pose controller: 1 "
                               "env x 4 robots x 10000 steps, a new goal pose on arrival within "
                               "0.05 m, fp32 (Table 2's pose-controller row)",
                          scenario=0, E=1, N=4, T=10000, precision=32, near=0.0, n_max=4,
                          goal_eps=0.05, episode_len=10000, controller=1,
                          context={"paper_table2_ms_per_10k_steps": 11.42,
                                   "paper_hardware": "JAX on an Apple M4 Pro CPU (pose "
                                                     "controller); another machine: context "
                                                     "only"}),
}


# the kernel each workload's rollout launches (one launch per bench step)
# 4-robot binary32 Navigation kernels by the tuner's variant (1 shuffle, 2 gather, 3 split)
NAV4_KERNELS = {1: "rl::env_kernel_small<1> (4-robot shuffle team kernel)",
                2: "rl::env_kernel_small<2> (4-robot gather team kernel)",
                3: "rl::env_kernel_split (4-robot shuffle teams, outputs in a second warp)"}
KERNELS = {"nav": "rl::env_kernel_small<1> (4-robot shuffle team kernel)",
           "waypoint": "rl::env_kernel_small<2> (4-robot gather team kernel)",
           "uneven": "rl::env_kernel_multi (one persistent launch over all size classes)",
           "largen": "rl::env_kernel<float, 32, 20> (20-robot class, explicit-inverse QP)",
           "tiny": "rl::env_kernel<double, 4, 4> (binary64 team kernel)",
           "waypoint_pose": "rl::env_kernel_small<2> (4-robot gather team kernel, pose controller)",
           "discovery": "rl::env_kernel_small<0> (4-robot general team kernel)"}


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="nav",
                   choices=list(WORKLOADS) + ["serving", "policy", "sweep"])
    p.add_argument("--hidden", type=int, default=128, help="policy: GRU width (App. A: 128-512)")
    p.add_argument("--duration", type=float, default=20.0, help="serving: seconds of arrivals")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    p.add_argument("--no-plain", action="store_true", help="skip the plain-form leg")
    p.add_argument("--no-tune", action="store_true", help="keep the default launch shape")
    p.add_argument("--variant", type=int, default=0,
                   help="4-robot Navigation: fix the kernel (1 shuffle, 2 gather, 3 split: the "
                        "tuner's pick on GB300) with the spread launch and skip the tuner, so "
                        "that runs under a profiler time the same kernel")
    p.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg")
    p.add_argument("--horizon", type=int, default=0,
                   help="override the workload's steps per rollout (small profiling cases)")
    return p.parse_args()


def _kernels_per_rollout(tuning) -> int:
    """Kernels one rollout launches: one (a single size class, or an uneven batch in one
    persistent launch), else one per size class (the per-class launch modes)."""
    if tuning and tuning.get("class_launch") in (0, 2) and len(tuning.get("classes", [])) > 1:
        return len(tuning["classes"])
    return 1


def _kernel_name(workload: str, tuning) -> str:
    """The kernel the rollout launches: the tuner's (or the fixed) 4-robot variant."""
    if workload == "waypoint_pose":
        return NAV4_KERNELS[2]  # the pose controller runs in the gather kernel only
    if tuning and workload in ("nav", "waypoint"):
        for c in tuning.get("classes", []) + ([tuning["fixed"]] if "fixed" in tuning else []):
            if c.get("nmax") == 4 and c.get("lanes") == 4 and c.get("variant") in NAV4_KERNELS:
                return NAV4_KERNELS[c["variant"]]
    return KERNELS.get(workload, "rl::env_kernel")


def _rank_seed(rank: int) -> int:
    """Each rank runs its own batch (weak scaling): the batch's seed."""
    return 1000 + rank


def _max_over_ranks(dist, ms: float, device) -> float:
    """The slowest rank's time, on every rank (the time itself with one rank)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_rate(units_per_rank: float, world: int, max_ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_rank * world / (max_ms / 1e3)


def _dist():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _code_only(text: str) -> str:
    """C++ source without its comments and blank space (what the compiler sees of it); string
    literals in the sources here hold no comment markers."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(ln.strip() for ln in text.splitlines() if ln.strip())


def _source_hash() -> str:
    """Hash of the CUDA library's code (comments excluded): a profile's counters hold for the
    kernels built from the source it names."""
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2505_06771_gb300", "csrc", "*"))):
        with open(f, encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def _ncu_traffic(workload: str, kernel: str = ""):
    """dram bytes per launch recorded from an ncu capture of this exact kernel source: the line
    for the kernel the rollout launched (traffic_bytes_per_launch[<kernel>]), else the
    workload's single line."""
    path = os.path.join(ROOT, "profiles", f"ncu_rollout_{workload}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    hm = re.search(r"source_hash:\s*([0-9a-f]+)", txt)
    if not hm or hm.group(1) != _source_hash():
        return None
    name = kernel.split(" ")[0]
    for km in re.finditer(r"traffic_bytes_per_launch\[([^\]]+)\]:\s*([0-9.eE+]+)", txt):
        if km.group(1) == name:
            return float(km.group(2))
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    return float(m.group(1)) if m else None


def _peaks(key: str = "hbm_gbs", fallback: float = 6800.0):
    """A measured peak (HBM GB/s, bf16 TFLOP/s) or the fallback figure."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        if key in d:
            return float(d[key]), "measured"
    return fallback, "fallback"


def _fp32_flops(w, n_robots, qp_iters: float, env_steps: float):
    """Algorithmic binary32 flops of Navigation env-steps (the method's arithmetic, counted from
    its formulas, not from the instructions a kernel executes): per robot 85 + 4 (N - 1)
    (projection 4, nominal velocity 4, two speed caps 12, noise 6, four arena rows 20, SI to
    unicycle 7, wheel clip 8, Euler step and heading wrap 9, new projected point 4, reward term
    11, relative poses of the observation 4 (N - 1)); per pair 21 (row 10, violation at u_nom 6,
    collision test 5); per env N + 2 (team reward); per active-set iteration a rescan of every
    row and the step, 6 P + 20 N + 8.  Square roots, sines and cosines are special-function
    calls, not counted.  Returns (flops, flops per env-step) or (None, None) for scenarios with
    resources."""
    import numpy as np
    if w["scenario"] != 0:
        return None, None
    N = np.asarray(n_robots, np.float64)
    P = N * (N - 1) / 2
    per_env = N * (85 + 4 * (N - 1)) + 21 * P + N + 2
    steps_per_env = env_steps / len(N)
    base = float(per_env.sum()) * steps_per_env
    it_cost = float((6 * P + 20 * N + 8).mean())
    flops = base + qp_iters * it_cost
    return flops, flops / env_steps


def _fp32_peak():
    """FP32 CUDA-core peak: SMs x 128 lanes x 2 (FMA) x the maximum SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz, src = _peaks("sm_max_mhz", 2070.0)
    return sms * 128 * 2 * mhz * 1e6 / 1e12, sms, mhz, src


class Clocks:
    """nvidia-smi samples (every 100 ms) around the timed region.  The sampler is streaming
    before the region starts (its first line is awaited, at most 3 s), every line is stamped on
    arrival, and the summary keeps the lines that arrived from the region's start to one
    interval after its end (a line reports the interval before it).  A region shorter than the
    interval may hold none: the first line after its start then stands for it, and
    `in_region` says so.  If no line came before the region (a sampler that buffers its output,
    or a slow start) the arrival times say nothing, and the summary takes every line
    (`in_region` null)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    INTERVAL_S = 0.1

    def __init__(self, index: int):
        self.index = index
        self.lines = []  # (host time of arrival, line)
        self.proc = None
        self.t0 = self.t1 = None
        self.streaming = False

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(int(self.INTERVAL_S * 1000))],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            self._wait_for(lambda: self.lines, 3.0)
            self.streaming = bool(self.lines)
        except (OSError, ValueError):
            self.proc = None
        self.t0 = time.perf_counter()
        return self

    def _wait_for(self, cond, limit_s: float):
        end = time.perf_counter() + limit_s
        while not cond() and time.perf_counter() < end and self.proc.poll() is None:
            time.sleep(0.005)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def __exit__(self, *exc):
        self.t1 = time.perf_counter()
        if self.proc:
            if self.streaming:
                # the line that reports the region's last interval
                self._wait_for(lambda: self.lines and self.lines[-1][0] > self.t1,
                               2 * self.INTERVAL_S + 0.05)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    @staticmethod
    def _parse(line: str):
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 7:
            return None
        try:
            return float(parts[0]), float(parts[1]), parts[3:7]
        except ValueError:
            return None

    def summary(self):
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        t0 = self.t0 if self.t0 is not None else float("-inf")
        t1 = self.t1 if self.t1 is not None else float("inf")
        stamped = [(t, self._parse(ln)) for t, ln in self.lines]
        stamped = [(t, v) for t, v in stamped if v is not None]
        if not self.streaming and self.t0 is not None:
            window, in_region = [v for _, v in stamped], None
        else:
            window = [v for t, v in stamped if t0 <= t <= t1 + self.INTERVAL_S]
            in_region = True
        if not window and in_region is not None:
            after = [v for t, v in stamped if t >= t0]
            window, in_region = after[:1], False
        if not window:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "in_region": None if in_region is None else False}
        reasons = set()
        for _, _, flags in window:
            for nm, v in zip(names, flags):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(v[0] for v in window),
                "sm_max_mhz": max(v[1] for v in window), "reasons": sorted(reasons),
                "samples": len(window), "in_region": in_region}


def _robots(w):
    from synth_inputs import uneven_robot_counts
    import numpy as np
    if w["N"] == "uneven":
        return uneven_robot_counts(0, w["E"], 2, 10)
    return np.full(w["E"], w["N"], np.int32)


def _cfg_overrides(w):
    return dict(n_max=w["n_max"], near_frac=w["near"], goal_eps=w.get("goal_eps", 0.0),
                episode_len=w.get("episode_len", 100), controller=w.get("controller", 0))


def _oracle_cfg(w):
    import oracle
    return oracle.default_cfg(w["scenario"], **_cfg_overrides(w))


def _cpu_baseline(w, budget_s: float = 20.0):
    """The FP64 oracle on the host cores: the workload in chunks of up to 100 steps, stopping
    after budget_s seconds; env-steps/s over the chunks done."""
    import oracle
    threads = os.cpu_count() or 1
    n = _robots(w)
    c = _oracle_cfg(w)
    s = oracle.reset(c, 0, n)
    chunk = min(100, w["T"])
    done_steps, t0 = 0, time.perf_counter()
    while done_steps < w["T"]:
        oracle.rollout(c, 0, s, chunk, want_obs=True, threads=threads)
        done_steps += chunk
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": w["E"] * done_steps / dt, "unit": "env-steps/s", "cores": threads,
            "kind": "oracle",
            "sample": f"{w['E']} envs x {done_steps} of {w['T']} steps of the same workload "
                      f"(FP64 C oracle, OpenMP over envs, observations written)"}


def run_reference(a):
    rank, world, _ = _dist()
    if rank != 0:
        return
    import oracle
    if a.workload not in WORKLOADS:
        print(json.dumps({"impl": "reference",
                          "unavailable": f"the {a.workload} workload has no oracle leg"}))
        return
    w = WORKLOADS[a.workload]
    threads = os.cpu_count() or 1
    n = _robots(w)
    c = _oracle_cfg(w)
    s = oracle.reset(c, 0, n)
    chunk = min(100, w["T"])  # env steps per bench step: E envs x chunk steps
    for _ in range(a.warmup):
        oracle.rollout(c, 0, s, min(10, chunk), want_obs=True, threads=threads)
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        oracle.rollout(c, 0, s, chunk, want_obs=True, threads=threads)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = w["E"] * chunk * a.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "env-steps/s",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * tot / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["desc"], "n_envs": w["E"],
                       "sample_per_step": f"{w['E']} envs x {chunk} steps"},
            "cpu_baseline": {"value": value, "unit": "env-steps/s", "cores": threads,
                             "kind": "oracle",
                             "sample": f"{w['E']} envs x {chunk} steps per bench step"},
            "e2e": {"value": value, "unit": "env-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _gpu_index(local):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            return int(vis.split(",")[local])
        except (ValueError, IndexError):
            pass
    return local


def _oracle_state(c, st):
    """oracle.State from a parsed GPU state blob (values widened exactly)."""
    import oracle
    s = oracle.State(c, st["n_robots"])
    for k in ("x", "y", "th", "gx", "gy", "gth"):
        getattr(s, k)[:] = st[k]
    s.level[:] = st["level"]
    s.t[:] = st["t"]
    s.ep[:] = st["ep"]
    s.n_res[:] = st["n_res"]
    if st["r_max"]:
        s.qx[:], s.qy[:] = st["qx"], st["qy"]
        s.qlevel[:], s.qactive[:] = st["qlevel"], st["qactive"]
    s.counters[:] = st["counters"].reshape(-1)
    return s


def _wrap(a):
    import numpy as np
    return (np.asarray(a) + np.pi) % (2 * np.pi) - np.pi


def _angle_columns(scenario, n_max):
    """Observation columns holding angles (compared on the circle)."""
    if scenario == 0:
        return [2] + [5 + 3 * s + 2 for s in range(n_max - 1)]
    if scenario == 2:
        return [2] + [5 + 5 * s + 2 for s in range(n_max - 1)]
    return [2] + [4 + 4 * s + 2 for s in range(n_max - 1)]


def _parity_sample(rl, w, env, seed, fdt, steps=3, trace_steps=8, trace_envs=64):
    """Part of the CPU-oracle leg: the FP64 oracle stepped from the timed handle's own states
    over the whole batch, against the timed launch (rl_rollout with T = 1: the tuned launch shape
    and its CUDA graph); then, on the first envs of a fresh handle, the filtered controls u*
    read back through the traced step against the oracle's."""
    import numpy as np
    import torch

    import oracle
    c = _oracle_cfg(w)
    E, R, od = env.n_envs, env.total_robots, env.obs_dim
    g_nmax = int(env.cfg["n_max"])
    obs = torch.empty(1, R, od, dtype=fdt, device="cuda")
    rew = torch.empty(1, E, dtype=fdt, device="cuda")
    done = torch.empty(1, E, dtype=torch.uint8, device="cuda")
    ep = eth = er = eo = 0.0
    exact = True
    for _ in range(steps):
        s = _oracle_state(c, env.state_arrays())
        obs_o, rew_o, done_o, _ = oracle.step(c, seed, s)
        env.rollout(1, obs, rew, done)
        torch.cuda.synchronize()
        st = env.state_arrays()
        exact &= bool(np.array_equal(done[0].cpu().numpy(), done_o))
        exact &= bool(np.array_equal(st["counters"][:, [0, 1, 2, 6]],
                                     s.counters.reshape(-1, 8)[:, [0, 1, 2, 6]]))
        if st["r_max"]:
            exact &= bool(np.array_equal(st["qactive"], s.qactive))
        ep = max(ep, float(np.abs(st["x"] - s.x).max()), float(np.abs(st["y"] - s.y).max()))
        eth = max(eth, float(np.abs(_wrap(st["th"] - s.th)).max()))
        er = max(er, float(np.abs(rew[0].cpu().numpy() - rew_o).max()))
        d = np.abs(obs[0].cpu().numpy().astype(np.float64) - obs_o)
        for col in _angle_columns(w["scenario"], g_nmax):
            d[:, col] = np.abs(_wrap(obs[0].cpu().numpy()[:, col].astype(np.float64) - obs_o[:, col]))
        eo = max(eo, float(d.max()) if d.size else 0.0)
    out = {"timed_launch": {"envs": E, "steps": steps, "integers_exact": exact,
                            "max_pose_err_per_step_m": ep, "max_heading_err_rad": eth,
                            "max_reward_err": er, "max_obs_err": eo,
                            "control_err_bound_from_pose": ep / float(w.get("dt", 0.033))}}
    n = _robots(w)[:trace_envs]
    g = rl.config_default(w["scenario"], precision=w["precision"], **_cfg_overrides(w))
    tenv = rl.Env(g, len(n), n, 0)
    us = torch.zeros(tenv.total_robots, 2, dtype=tenv.dtype, device="cuda")
    qi = torch.zeros(len(n), 4, dtype=torch.int32, device="cuda")
    eu = epp = 0.0
    flagged = 0
    for _ in range(trace_steps):
        s = _oracle_state(c, tenv.state_arrays())
        _, _, _, tr = oracle.step(c, 0, s, trace=True)
        tenv.step(u_star=us, qp_info=qi)
        st2 = tenv.state_arrays()
        eu = max(eu, float(np.abs(us.cpu().numpy() - tr["u_star"]).max()))
        epp = max(epp, float(np.abs(st2["x"] - s.x).max()), float(np.abs(st2["y"] - s.y).max()))
        flagged += int(((qi.cpu().numpy()[:, 3] >> 1) & 1).sum())
    tenv.close()
    out["traced_step"] = {"envs": len(n), "steps": trace_steps, "max_control_err": eu,
                          "max_pose_err_per_step_m": epp, "fp64_resolved": flagged}
    out["tolerances"] = {"control": 1e-5, "pose_per_step_m": 3e-7, "reward": 1e-5, "obs": 1e-5}
    return out


def run_rollout(a):
    import numpy as np
    import torch

    import paper_2505_06771_gb300 as rl

    rank, world, local = _dist()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    rl.lib()
    w = dict(WORKLOADS[a.workload])
    if a.horizon > 0:
        w["T"] = a.horizon
        w["desc"] += f" (horizon overridden: {a.horizon} steps)"
    E, T = w["E"], w["T"]
    n = _robots(w)
    stream = torch.cuda.Stream()
    g = rl.config_default(w["scenario"], precision=w["precision"], **_cfg_overrides(w))
    if a.variant:
        g.update(small_variant=a.variant, block_threads=128, warp_envs=0)
    fdt = torch.float64 if w["precision"] == 64 else torch.float32
    esz = 8 if w["precision"] == 64 else 4
    with torch.cuda.stream(stream):
        env = rl.Env(g, E, n, seed=_rank_seed(rank), stream=stream)
        rows = env.total_robots
        obs = torch.empty(T, rows, env.obs_dim, dtype=fdt, device="cuda")
        rew = torch.empty(T, E, dtype=fdt, device="cuda")
        done = torch.empty(T, E, dtype=torch.uint8, device="cuda")
    stream.synchronize()
    tuning = None
    if a.variant:
        tuning = {"fixed": {"nmax": 4, "lanes": 4, "block_threads": 128, "warp_envs": 0,
                            "variant": a.variant}}
    elif not a.no_tune and w["precision"] == 32:
        # probes of up to 1000 steps: the slow tail of a rollout (a few envs whose robots stay
        # jammed for many steps) decides its time and does not show in short probes
        tuning = env.tune(min(1000, T))
    n_warm = max(3, a.warmup)
    for _ in range(n_warm):
        env.rollout(T, obs, rew, done)
    stream.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(a.steps)]
    with Clocks(_gpu_index(local)) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(a.steps):
            ev[i][0].record(stream)
            env.rollout(T, obs, rew, done)
            ev[i][1].record(stream)
        t_end.record(stream)
        stream.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
    total_ms = t_start.elapsed_time(t_end)
    per = [s.elapsed_time(e) for s, e in ev]
    counters = env.counters()  # since the tuner: the warm-up and timed rollouts
    env_steps_counted = E * T * (n_warm + a.steps)
    total_ms = _max_over_ranks(dist, total_ms, "cuda")
    value = _job_rate(E * T * a.steps, world, total_ms)

    # ---- roofline of the rollout kernel (the only kernel of the step)
    traj_bytes = T * (rows * env.obs_dim * esz + E * esz + E)
    state_bytes = 2 * (rows * (5 * esz + 4) + E * (3 * 4 + 8 * 4))
    alg_bytes = traj_bytes + state_bytes
    kernel_ms = statistics.mean(per)
    achieved = alg_bytes / (kernel_ms / 1e3) / 1e9
    peak, peak_src = _peaks()
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak,
            "traffic": _ncu_traffic(a.workload, _kernel_name(a.workload, tuning)),
            "peak_source": peak_src, "kernel": _kernel_name(a.workload, tuning),
            "algorithmic_bytes_per_launch": alg_bytes,
            "bytes_per_env_step": alg_bytes / (E * T)}

    # ---- the same kernel against the FP32 CUDA-core peak (algorithmic flops, with the active-set
    # iterations the counters recorded over the warm-up and timed rollouts)
    iters_per_env_step = float(counters[:, 7].sum()) / env_steps_counted
    fl, fl_es = _fp32_flops(w, n, iters_per_env_step * E * T, E * T)
    if fl is not None:
        pk, sms, mhz, src = _fp32_peak()
        ach = fl / (kernel_ms / 1e3) / 1e12
        roof_fp32 = {"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                     "frac": ach / pk, "flops_per_env_step": fl_es,
                     "qp_iters_per_env_step": iters_per_env_step,
                     "peak_source": f"{sms} SMs x 128 x 2 x {mhz:.0f} MHz ({src} max SM clock)"}
    else:
        roof_fp32 = None

    extra = {}
    if not a.no_plain and a.workload == "nav":
        Tp = 2
        po = torch.empty(Tp, rows, env.obs_dim, dtype=fdt, device="cuda")
        pr = torch.empty(Tp, E, dtype=fdt, device="cuda")
        pd = torch.empty(Tp, E, dtype=torch.uint8, device="cuda")
        env.rollout(1, po, pr, pd, plain=True)
        stream.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        env.rollout(Tp, po, pr, pd, plain=True)
        s1.record(stream)
        stream.synchronize()
        pv = E * Tp / (s0.elapsed_time(s1) / 1e3)
        extra["plain_form"] = {"value": pv, "unit": "env-steps/s",
                               "sample": f"{Tp} steps x {E} launches per step"}
        extra["speedup_vs_plain"] = value / world / pv

    # ---- end to end through host buffers (state upload + trajectory download per step)
    e2e = None
    if not a.no_e2e:
        blob = np.frombuffer(env.get_state(), np.uint8).copy()
        h_state = torch.from_numpy(blob).pin_memory()
        h_obs = torch.empty(T, rows, env.obs_dim, dtype=fdt, pin_memory=True)
        h_rew = torch.empty(T, E, dtype=fdt, pin_memory=True)
        h_done = torch.empty(T, E, dtype=torch.uint8, pin_memory=True)
        env.rollout_host(T, h_state.numpy(), h_obs, h_rew, h_done)  # warm-up
        K2 = max(2, min(a.steps, 5))
        t0 = time.perf_counter()
        for _ in range(K2):
            env.rollout_host(T, h_state.numpy(), h_obs, h_rew, h_done)
        e2e_s = (time.perf_counter() - t0) / K2
        e2e = {"value": E * T * world / e2e_s, "unit": "env-steps/s",
               "h2d_bytes_per_step": int(blob.nbytes),
               "d2h_bytes_per_step": int(h_obs.numel() * esz + h_rew.numel() * esz +
                                         h_done.numel())}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": world,
                "steps": a.steps, "warmup": max(3, a.warmup), "ms_per_step": total_ms / a.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if w["precision"] == 64 else "f32", "data": "synthetic",
                "config": {"workload": w["desc"], "n_envs": E,
                           "n_robots": w["N"] if w["N"] != "uneven" else "U{2..10}",
                           "total_robots": rows, "horizon": T,
                           "episode_len": w.get("episode_len", 100),
                           "obs": f"[{T}, {rows}, {env.obs_dim}] per step",
                           "l2": f"trajectory outputs of {traj_bytes / 1e6:.0f} MB per step "
                                 "(larger than the 129 MB L2 except for the tiny workload)",
                           "parallelism": f"{world} GPU(s), envs independent per rank",
                           "tuning": tuning},
                "robot_steps_per_s": value * rows / E,
                "latency_ms": {"p50": float(np.percentile(per, 50)),
                               "p99": float(np.percentile(per, 99))},
                "roofline": roof, "roofline_fp32": roof_fp32, "e2e": e2e,
                "gpu_launches": a.steps * _kernels_per_rollout(tuning),
                "clocks": clk.summary(),
                "qp": {"active_step_frac": float(counters[:, 3].sum()) / env_steps_counted,
                       "fp64_resolved_frac": float(counters[:, 4].sum()) / env_steps_counted,
                       "collisions": int(counters[:, 0].sum())}}
        if w.get("goal_eps"):
            line["waypoint_arrivals_per_10k_steps"] = \
                1e4 * float(counters[:, 2].sum()) / env_steps_counted
        if "context" in w:
            line["context"] = w["context"]
        line.update(extra)
        if world == 1 and not a.no_cpu:
            # the CPU-oracle leg: the oracle timed on the host cores, and the oracle's results
            # against the timed launch's on the same states (max error per result)
            line["cpu_baseline"] = _cpu_baseline(w)
            line["parity_sample"] = _parity_sample(rl, w, env, _rank_seed(rank), fdt)
        print(json.dumps(line), flush=True)
    env.close()
    if dist:
        dist.destroy_process_group()


def run_serving(a):
    """Poisson arrivals (200 req/s) of rollout requests: n_envs log-uniform in [1, 2048], robots
    uniform in {2..12}, horizon uniform in [100, 1000]; 60 GB budget; p50/p99 latency."""
    import numpy as np
    import torch

    import paper_2505_06771_gb300 as rl
    from synth_inputs import serving_requests

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if rank != 0 and world > 1:
        pass
    g = rl.config_default(0, n_max=12)
    srv = rl.Server(g, 60 << 30, 32)
    reqs = serving_requests(100 + rank, a.duration, rate_hz=200.0)
    warm = srv.submit(64, 4, 100, 1)
    srv.drain(60.0)
    srv.result(warm)
    ids = []
    with Clocks(_gpu_index(local)) as clk:
        t0 = time.perf_counter()
        for q in reqs:
            dt = q["arrival_s"] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            ids.append(srv.submit(q["n_envs"], q["n_robots"], q["horizon"], q["seed"]))
        ok = srv.drain(600.0)
        wall = time.perf_counter() - t0
    res = [srv.result(i) for i in ids]
    st = srv.stats()
    srv.close()
    lat = np.array([r["latency_s"] for r in res if r["status"] == 2]) * 1e3
    wait = np.array([r["start_s"] - r["submit_s"] for r in res if r["status"] == 2]) * 1e3
    env_steps = sum(r["n_envs"] * r["horizon"] for r in res if r["status"] == 2)
    robot_steps = sum(r["n_envs"] * r["horizon"] * r["n_robots"] for r in res if r["status"] == 2)
    line = {"metric": METRIC, "value": env_steps / wall, "unit": "env-steps/s", "n_gpus": world,
            "steps": len(reqs), "warmup": 1, "ms_per_step": 1e3 * wall / max(1, len(reqs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "serving: Poisson 200 req/s, n_envs log-U[1,2048], robots "
                                   "U{2..12}, horizon U[100,1000], 60 GB budget, 32 slots",
                       "duration_s": a.duration, "requests": len(reqs)},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "mean": float(lat.mean())},
            "queue_wait_ms": {"p50": float(np.percentile(wait, 50)),
                              "p99": float(np.percentile(wait, 99))},
            "robot_steps_per_s": robot_steps / wall, "completed": int(len(lat)),
            "drained": bool(ok), "peak_bytes": st["peak"], "clocks": clk.summary(),
            "gpu_launches": len(reqs)}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_policy(a):
    """Policy in the loop: Navigation 4096 envs x 4 robots x 1000 steps driven by an MLP -> GRU
    -> linear policy evaluated on the GPU between steps (one tensor-core kernel per step)."""
    import numpy as np
    import torch

    import paper_2505_06771_gb300 as rl
    from synth_inputs import policy_weights

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    E, N, T, H = 4096, 4, (a.horizon or 1000), a.hidden
    stream = torch.cuda.Stream()
    g = rl.config_default(0, scripted=0, n_max=N)
    with torch.cuda.stream(stream):
        env = rl.Env(g, E, N, seed=_rank_seed(rank), stream=stream)
        R, od = env.total_robots, env.obs_dim
        pol = rl.Policy(env, policy_weights(7, H, od))
        obs0 = torch.empty(R, od, device="cuda")
        obs = torch.empty(T, R, od, device="cuda")
        rew = torch.empty(T, E, device="cuda")
        done = torch.empty(T, E, dtype=torch.uint8, device="cuda")
    env.observe(obs0)
    stream.synchronize()
    n_warm = max(3, a.warmup)
    for _ in range(n_warm):
        pol.rollout(T, obs0, obs, done, reward=rew)
    stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(a.steps)]
    with Clocks(_gpu_index(local)) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(a.steps):
            ev[i][0].record(stream)
            pol.rollout(T, obs0, obs, done, reward=rew)
            ev[i][1].record(stream)
        t1.record(stream)
        stream.synchronize()
    total_ms = t0.elapsed_time(t1)
    per = [s.elapsed_time(e) for s, e in ev]
    value = E * T * a.steps / (total_ms / 1e3)
    # the products of every step, algorithmic (no zero blocks): h1 = W1 o (K = 16, the
    # observation padded), r and z over K = 2H, n_i and n_h over K = H each
    flops = 2.0 * T * R * (16 * H + 6 * H * H)
    peak, src = _peaks(key="bf16_tflops_sustained", fallback=1700.0)
    achieved = flops / (statistics.mean(per) / 1e3) / 1e12
    line = {"metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": 1,
            "steps": a.steps, "warmup": n_warm, "ms_per_step": total_ms / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16",
            "data": "synthetic",
            "config": {"workload": f"policy in the loop: navigation {E} envs x {N} robots x {T} "
                                   f"steps, MLP(ReLU, {H}) -> GRU({H}) -> linear policy between "
                                   "steps (one hand-written tcgen05 kernel per policy step, "
                                   "bf16 operands, binary32 accumulators in tensor memory)",
                       "n_envs": E, "horizon": T, "hidden": H},
            "latency_ms": {"p50": float(np.percentile(per, 50)),
                           "p99": float(np.percentile(per, 99))},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None, "peak_source": src,
                         "kernel": "rl::ptc::policy_step_tc (the policy's products), flops "
                                   "over the whole rollout time (policy and environment kernels)",
                         "flops_per_rollout": flops},
            "e2e": None, "gpu_launches": 2 * T * a.steps, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    pol.close()
    env.close()


SWEEP_ENVS = (1, 16, 128, 1024, 4096, 16384, 65536)


def run_sweep(a):
    """Navigation, 4 robots, 1000-step rollouts (10 episodes) at each number of environments
    in SWEEP_ENVS, each launch shape picked by the autotuner: env-steps/s and ms per rollout
    (mean of --steps rollouts after the warm-ups).  The paper measures the same scaling with
    JAX on a CPU (Sec. 4.2, Fig. 2: 100K timesteps over a range of environment counts); its
    values are in a figure only, so there is no number to compare with."""
    import torch

    import paper_2505_06771_gb300 as rl

    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device")
    rank, world, local = _dist()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    rl.lib()
    T = a.horizon if a.horizon > 0 else 1000
    w = dict(WORKLOADS["nav"])
    stream = torch.cuda.Stream()
    rows_out = []
    launches = 0
    with Clocks(_gpu_index(local)) as clk:
        for E in SWEEP_ENVS:
            g = rl.config_default(0, precision=32, **_cfg_overrides(w))
            with torch.cuda.stream(stream):
                env = rl.Env(g, E, 4, seed=_rank_seed(0), stream=stream)
                obs = torch.empty(T, E * 4, env.obs_dim, device="cuda")
                rew = torch.empty(T, E, device="cuda")
                done = torch.empty(T, E, dtype=torch.uint8, device="cuda")
            stream.synchronize()
            tuning = env.tune(min(T, 500)) if not a.no_tune else None
            for _ in range(max(3, a.warmup)):
                env.rollout(T, obs, rew, done)
            stream.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(a.steps)]
            for i in range(a.steps):
                ev[i][0].record(stream)
                env.rollout(T, obs, rew, done)
                ev[i][1].record(stream)
            stream.synchronize()
            launches += a.steps
            per = [s_.elapsed_time(e_) for s_, e_ in ev]
            ms = statistics.mean(per)
            rows_out.append({"n_envs": E, "ms_per_rollout": ms, "env_steps_per_s": E * T / (ms / 1e3),
                             "robot_steps_per_s": 4 * E * T / (ms / 1e3),
                             "p99_ms": sorted(per)[min(len(per) - 1, int(0.99 * len(per)))],
                             "tuning": tuning})
            env.close()
            del obs, rew, done
            torch.cuda.empty_cache()
    best = max(r["env_steps_per_s"] for r in rows_out)
    line = {"metric": METRIC, "value": best, "unit": "env-steps/s", "n_gpus": 1, "steps": a.steps,
            "warmup": max(3, a.warmup), "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"navigation sweep over n_envs {list(SWEEP_ENVS)} x 4 robots x "
                                   f"{T} steps, scripted nominal control, fp32",
                       "l2": "trajectory outputs larger than L2 from 1024 envs on"},
            "sweep": rows_out, "gpu_launches": launches, "clocks": clk.summary(),
            "context": {"paper": "Sec. 4.2, Fig. 2: JAX on an Apple M4 Pro CPU, values in a "
                                 "figure only (another machine: context, not a target)"}}
    print(json.dumps(line), flush=True)


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "serving":
        run_serving(a)
    elif a.workload == "policy":
        run_policy(a)
    elif a.workload == "sweep":
        run_sweep(a)
    else:
        run_rollout(a)


if __name__ == "__main__":
    main()
