"""Serving (continuous batching) on the GPU: results are the same alone and in a mix of
requests admitted at different times, admission respects the memory budget, and waits are
bounded."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2505_06771_gb300 as m
    m.build()
    return m


def test_result_same_alone_and_in_the_mix(rl):
    from synth_inputs import serving_requests
    g = rl.config_default(0)
    probe = dict(n_envs=300, n_robots=7, horizon=250, seed=987654321)
    alone = rl.Server(g, 8 << 30, 4)
    rid = alone.submit(**probe)
    assert alone.drain(60.0)
    ref = alone.result(rid, returns=True)
    alone.close()
    assert ref["status"] == 2

    mix = rl.Server(g, 8 << 30, 6)
    reqs = serving_requests(3, 0.25, rate_hz=200.0, envs_max=512, horizon_hi=400)
    ids = []
    t0 = time.perf_counter()
    for k, q in enumerate(reqs):
        while time.perf_counter() - t0 < q["arrival_s"]:
            time.sleep(0.0005)
        ids.append(mix.submit(q["n_envs"], q["n_robots"], q["horizon"], q["seed"]))
        if k == len(reqs) // 2:
            pid = mix.submit(**probe)
    assert mix.drain(120.0)
    got = mix.result(pid, returns=True)
    st = mix.stats()
    mix.close()
    assert got["status"] == 2
    assert np.array_equal(got["returns"], ref["returns"])
    assert got["counters"] == ref["counters"]
    assert st["done"] == len(reqs) + 1
    print(f"\nmix of {len(reqs) + 1} requests; probe latency {got['latency_s'] * 1e3:.2f} ms")


def test_budget_bounds_admission(rl):
    g = rl.config_default(0)
    need = 2 * 1024 * (5 * 4 * 8 + 300)  # about two of the requests below
    srv = rl.Server(g, need, 8)
    with pytest.raises(rl.RLError) as ei:
        srv.submit(100000, 8, 10, 1)  # can never fit
    assert ei.value.status == 6
    ids = [srv.submit(1024, 8, 300, s) for s in range(6)]
    assert srv.drain(60.0)
    st = srv.stats()
    assert st["peak"] <= need and st["used"] == 0 and st["done"] == 6
    assert all(srv.result(i)["status"] == 2 for i in ids)
    srv.close()


def test_drain_timeout_is_bounded(rl):
    g = rl.config_default(0)
    srv = rl.Server(g, 8 << 30, 2)
    srv.submit(2048, 12, 1000, 5)
    t0 = time.perf_counter()
    finished = srv.drain(0.0005)
    waited = time.perf_counter() - t0
    assert waited < 0.5
    assert srv.drain(120.0)
    srv.close()
    assert finished in (True, False)
