"""Host logic of the benchmark (CPU): the source hash that ties a profile's DRAM counters to the
kernels they were taken on, the per-kernel lookup of those counters, the launch count, the
clock-sample summary, the peak lookup and the algorithmic binary32 flop count."""
import bench


def test_code_only_drops_comments_and_blank_space():
    src = "int a; // a comment\n/* block\n comment */\n\n   int b = 2;  \n"
    assert bench._code_only(src) == "int a;\nint b = 2;"
    # a code change shows, a comment change does not
    assert bench._code_only("x = 1; // one") == bench._code_only("x = 1; // uno")
    assert bench._code_only("x = 1;") != bench._code_only("x = 2;")


def test_ncu_traffic_per_kernel_and_source(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    csrc = tmp_path / "paper_2505_06771_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("__global__ void k() {}  // v1\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = bench._source_hash()
    (prof / "ncu_rollout_nav.md").write_text(
        "traffic_bytes_per_launch[rl::kern_a]: 100\n"
        "traffic_bytes_per_launch[rl::kern_b<1>]: 200\n"
        f"source_hash: {h}\n")
    assert bench._ncu_traffic("nav", "rl::kern_a (the first kernel)") == 100.0
    assert bench._ncu_traffic("nav", "rl::kern_b<1> (another)") == 200.0
    assert bench._ncu_traffic("nav", "rl::kern_c (not captured)") is None
    assert bench._ncu_traffic("largen", "rl::kern_a") is None  # no profile
    # a comment edit keeps the capture, a code edit voids it
    (csrc / "k.cu").write_text("__global__ void k() {}  // v2, reworded\n")
    assert bench._ncu_traffic("nav", "rl::kern_a (x)") == 100.0
    (csrc / "k.cu").write_text("__global__ void k() { int x = 0; }\n")
    assert bench._ncu_traffic("nav", "rl::kern_a (x)") is None
    # a profile with a single kernel's line
    (prof / "ncu_rollout_nav.md").write_text(
        f"traffic_bytes_per_launch: 300\nsource_hash: {bench._source_hash()}\n")
    assert bench._ncu_traffic("nav", "rl::anything") == 300.0


def test_kernels_per_rollout():
    assert bench._kernels_per_rollout(None) == 1
    one = dict(nmax=4, lanes=4, block_threads=128, warp_envs=0, variant=3)
    assert bench._kernels_per_rollout({"fixed": one}) == 1
    three = [dict(one, nmax=n) for n in (4, 8, 16)]
    assert bench._kernels_per_rollout({"class_launch": 1, "classes": three}) == 1
    assert bench._kernels_per_rollout({"class_launch": 0, "classes": three}) == 3
    assert bench._kernels_per_rollout({"class_launch": 2, "classes": three}) == 3
    assert bench._kernels_per_rollout({"class_launch": 0, "classes": three[:1]}) == 1


def test_clock_summary_median_max_and_reasons():
    c = bench.Clocks(0)
    c.t0, c.t1, c.streaming = 10.0, 10.5, True
    c.lines = [(9.9, "1200, 2070, 300.0, Not Active, Not Active, Not Active, Not Active"),  # before
               (10.1, "2070, 2070, 900.1, Not Active, Not Active, Not Active, Not Active"),
               (10.3, "1980, 2070, 1390.0, Not Active, Not Active, Not Active, Active"),
               (10.55, "2070, 2070, 1201.0, Not Active, Not Active, Not Active, Not Active"),
               (10.58, "[N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]"),  # unreadable
               (10.59, "garbage"),
               (10.9, "210, 2070, 100.0, Active, Not Active, Not Active, Not Active")]  # after
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3, "in_region": True}
    c.lines = [(10.2, "1500, 2070, 700, Active, Not Active, Active, Not Active")]
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    # a region shorter than the sampling interval: the first line after its start stands for it
    c.t0, c.t1 = 10.0, 10.01
    c.lines = [(9.95, "1000, 2070, 1, Not Active, Not Active, Not Active, Not Active"),
               (10.2, "2055, 2070, 1, Not Active, Not Active, Not Active, Not Active"),
               (10.3, "900, 2070, 1, Not Active, Not Active, Not Active, Not Active")]
    s = c.summary()
    assert s["sm_mhz"] == 2055.0 and s["samples"] == 1 and s["in_region"] is False
    c.lines = []
    assert c.summary()["samples"] == 0 and c.summary()["sm_mhz"] is None
    # a sampler whose lines came only after the region (buffered output): every line counts
    c.streaming = False
    c.lines = [(11.0, "2070, 2070, 1, Not Active, Not Active, Not Active, Not Active"),
               (11.0, "2040, 2070, 1, Not Active, Not Active, Not Active, Active")]
    s = c.summary()
    assert s["samples"] == 2 and s["in_region"] is None and s["sm_mhz"] == 2055.0
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_sampler_streams_through_the_region(tmp_path, monkeypatch):
    # a stand-in nvidia-smi that prints one sample every 20 ms after a start-up delay
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/usr/bin/env python3\n"
                    "import sys, time\n"
                    "time.sleep(0.2)\n"
                    "while True:\n"
                    "    print('2070, 2070, 800.0, Not Active, Not Active, Not Active, Not Active',"
                    " flush=True)\n"
                    "    time.sleep(0.02)\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + ":" + __import__("os").environ["PATH"])
    with bench.Clocks(0) as c:
        assert c.lines, "the sampler streams before the region starts"
        import time
        time.sleep(0.3)
    s = c.summary()
    assert c.streaming and s["in_region"] and s["samples"] >= 5 and s["sm_mhz"] == 2070.0
    assert c.proc.poll() is not None  # stopped
    # no nvidia-smi at all: an empty summary, no wait
    monkeypatch.setenv("PATH", str(tmp_path / "none"))
    with bench.Clocks(0) as c:
        pass
    assert c.summary()["samples"] == 0


def test_peaks_measured_or_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._peaks("hbm_gbs", 6800.0) == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6780.4, "bf16_tflops": 1988}')
    assert bench._peaks("hbm_gbs", 6800.0) == (6780.4, "measured")
    assert bench._peaks("bf16_tflops_sustained", 1700.0) == (1700.0, "fallback")


def test_fp32_flops_per_env_step():
    # 4 robots: per robot 85 + 4 * 3, per pair 21 (6 pairs), per env 4 + 2 -> 520 flops per
    # env-step without active-set iterations; an iteration rescans 6 pair and 16 arena rows: 124
    flops, per = bench._fp32_flops({"scenario": 0}, [4] * 10, qp_iters=0.0, env_steps=10)
    assert flops == 5200.0 and per == 520.0
    flops, per = bench._fp32_flops({"scenario": 0}, [4] * 10, qp_iters=3.2, env_steps=10)
    assert abs(per - (520.0 + 0.32 * 124.0)) < 1e-9
    # 20 robots: 20 * (85 + 76) + 21 * 190 + 22 = 7232
    assert bench._fp32_flops({"scenario": 0}, [20], 0.0, 1)[1] == 7232.0
    assert bench._fp32_flops({"scenario": 1}, [4], 0.0, 1) == (None, None)
