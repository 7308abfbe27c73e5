#!/usr/bin/env python
"""Benchmark of the batched CBF-QP multi-robot environment step on GB300.

Workload (one bench step): the Navigation batch of 4096 environments x 4 robots, 1000 scripted
steps (10 episodes of 100 steps), binary32, run by rl_rollout as one CUDA-graph replay of the
persistent kernel, streaming observations [1000, 16384, 14], rewards and done flags (938 MB)
to HBM.  Reported: env-steps/s (and robot-steps/s), the plain one-launch-per-env-per-step form
of the same step, p50/p99 rollout latency, the HBM roofline fraction of the rollout kernel, the
end-to-end rate through host buffers, and the FP64 CPU oracle timed on the host cores.

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
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
E, N, T = 4096, 4, 1000
WORKLOAD = "navigation: 4096 envs x 4 robots x 1000 steps, scripted nominal control, fp32"


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    p.add_argument("--no-plain", action="store_true", help="skip the plain-form leg")
    return p.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _source_hash() -> str:
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2505_06771_gb300", "csrc", "*"))):
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic():
    """dram bytes per launch recorded from an ncu capture of this exact kernel source."""
    path = os.path.join(ROOT, "profiles", "ncu_rollout_nav4096x4.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    hm = re.search(r"source_hash:\s*([0-9a-f]+)", txt)
    if not m or not hm or hm.group(1) != _source_hash():
        return None
    return float(m.group(1))


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh).get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _cpu_baseline(budget_s: float = 20.0):
    """The FP64 oracle on the host cores: up to the full workload in 100-step chunks, stopping
    after budget_s seconds; env-steps/s over the chunks done."""
    import oracle
    threads = os.cpu_count() or 1
    c = oracle.default_cfg(oracle.NAV, n_max=N)
    s = oracle.reset(c, 0, [N] * E)
    done_steps, t0 = 0, time.perf_counter()
    while done_steps < T:
        oracle.rollout(c, 0, s, 100, want_obs=True, threads=threads)
        done_steps += 100
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": E * done_steps / dt, "unit": "env-steps/s", "cores": threads,
            "kind": "oracle",
            "sample": f"{E} envs x {N} robots x {done_steps} steps of the same workload "
                      f"(FP64 C oracle, OpenMP over envs, observations written)"}


def run_reference(a):
    rank, world, _ = _dist()
    if rank != 0:
        return
    import oracle
    threads = os.cpu_count() or 1
    c = oracle.default_cfg(oracle.NAV, n_max=N)
    s = oracle.reset(c, 0, [N] * E)
    chunk = 100  # env steps per bench step: 4096 envs x 100 steps
    for _ in range(a.warmup):
        oracle.rollout(c, 0, s, 10, want_obs=True, threads=threads)
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        oracle.rollout(c, 0, s, chunk, want_obs=True, threads=threads)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = E * chunk * a.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "env-steps/s",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * tot / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_envs": E, "n_robots": N,
                       "sample_per_step": f"{E} envs x {chunk} steps"},
            "cpu_baseline": {"value": value, "unit": "env-steps/s", "cores": threads,
                             "kind": "oracle",
                             "sample": f"{E} envs x {N} robots x {chunk} steps per bench step"},
            "e2e": {"value": value, "unit": "env-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(a):
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
    stream = torch.cuda.Stream()
    g = rl.config_default(rl.NAVIGATION)
    with torch.cuda.stream(stream):
        env = rl.Env(g, E, N, seed=1000 + rank, stream=stream)
        rows = env.total_robots
        obs = torch.empty(T, rows, env.obs_dim, device="cuda")
        rew = torch.empty(T, E, device="cuda")
        done = torch.empty(T, E, dtype=torch.uint8, device="cuda")
    stream.synchronize()

    for _ in range(max(3, a.warmup)):
        env.rollout(T, obs, rew, done)
    stream.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(a.steps)]
    gpu_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            gpu_index = int(vis.split(",")[local])
        except ValueError:
            pass
    with Clocks(gpu_index) as clk:
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
    if dist:
        tt = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    env_steps = E * T * a.steps * world
    value = env_steps / (total_ms / 1e3)

    # ---- roofline of the rollout kernel (the only kernel of the step)
    bytes_per_env_step = 4 * N * env.obs_dim + 4 + 1
    state_bytes = rows * (5 * 4 * 2 + 4 * 2) + E * (4 * 2 * 2 + 8 * 4 * 2)
    alg_bytes = E * T * bytes_per_env_step + state_bytes
    kernel_ms = statistics.mean(per)
    achieved = alg_bytes / (kernel_ms / 1e3) / 1e9
    peak, peak_src = _peaks()
    traffic = _ncu_traffic()
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
            "kernel": "rl::env_kernel<float, lanes, 4>",
            "bytes_per_env_step": bytes_per_env_step}

    extra = {}
    # ---- plain one-launch-per-env-per-step form (bounded sample)
    if not a.no_plain:
        Tp = 2
        po = torch.empty(Tp, rows, env.obs_dim, device="cuda")
        pr = torch.empty(Tp, E, device="cuda")
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
    blob = np.frombuffer(env.get_state(), np.uint8).copy()
    h_state = torch.from_numpy(blob).pin_memory()
    h_obs = torch.empty(T, rows, env.obs_dim, pin_memory=True)
    h_rew = torch.empty(T, E, pin_memory=True)
    h_done = torch.empty(T, E, dtype=torch.uint8, pin_memory=True)
    env.rollout_host(T, h_state.numpy(), h_obs, h_rew, h_done)  # warm-up
    K2 = max(2, min(a.steps, 5))
    t0 = time.perf_counter()
    for _ in range(K2):
        env.rollout_host(T, h_state.numpy(), h_obs, h_rew, h_done)
    e2e_s = (time.perf_counter() - t0) / K2
    e2e = {"value": E * T * world / e2e_s, "unit": "env-steps/s",
           "h2d_bytes_per_step": int(blob.nbytes),
           "d2h_bytes_per_step": int(h_obs.numel() * 4 + h_rew.numel() * 4 + h_done.numel())}

    counters = env.counters()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": world,
                "steps": a.steps, "warmup": max(3, a.warmup), "ms_per_step": total_ms / a.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "scenario": "navigation", "n_envs": E,
                           "n_robots": N, "horizon": T, "episode_len": 100,
                           "obs": f"[{T}, {rows}, {env.obs_dim}] f32 per step",
                           "l2": "trajectory outputs of 938 MB per step exceed the 129 MB L2",
                           "parallelism": f"{world} GPU(s), envs independent per rank",
                           "lanes_per_env": env.lanes},
                "robot_steps_per_s": value * N,
                "latency_ms": {"p50": float(np.percentile(per, 50)),
                               "p99": float(np.percentile(per, 99))},
                "roofline": roof, "e2e": e2e, "gpu_launches": a.steps,
                "clocks": clk.summary(),
                "qp": {"active_step_frac": float(counters[:, 3].sum()) / max(1, counters[:, 6].sum() * 100),
                       "fp64_resolved": int(counters[:, 4].sum()),
                       "collisions": int(counters[:, 0].sum())}}
        line.update(extra)
        if world == 1 and not a.no_cpu:
            line["cpu_baseline"] = _cpu_baseline()
        print(json.dumps(line), flush=True)
    env.close()
    if dist:
        dist.destroy_process_group()


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
