"""Host logic of the benchmark (CPU): the source hash that ties a profile's DRAM counters to the
kernels they were taken on, and the per-kernel lookup of those counters."""
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
