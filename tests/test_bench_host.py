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
    c.lines = ["2070, 2070, 900.1, Not Active, Not Active, Not Active, Not Active",
               "1980, 2070, 1390.0, Not Active, Not Active, Not Active, Active",
               "2070, 2070, 1201.0, Not Active, Not Active, Not Active, Not Active",
               "[N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",  # unreadable sample: skipped
               "garbage"]
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3}
    c.lines = ["1500, 2070, 700, Active, Not Active, Active, Not Active"]
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    c.lines = []
    assert c.summary()["samples"] == 0 and c.summary()["sm_mhz"] is None


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
