"""The benchmark's multi-GPU path (replicas, weak scaling) with world_size 2 on CPU (gloo):
every rank gets the slowest rank's time, the whole-job rate counts every rank's units, ranks
run different batches, and the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [10.0, 12.5][rank]
    dist.barrier()
    m = bench._max_over_ranks(dist, local_ms, "cpu")
    out[rank] = (m, bench._job_rate(4096 * 1000, world, m), bench._rank_seed(rank),
                 bench._dist())
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_time_and_job_rate():
    world, port = 2, _free_port()
    # the manager process is spawned too: forking this (multi-threaded) process could deadlock
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        m, rate, seed, d = res[rank]
        assert m == 12.5                                  # the slowest rank, on every rank
        assert abs(rate - 2 * 4096 * 1000 / 0.0125) < 1e-6
        assert d == (rank, world, rank)
    assert res[0][2] != res[1][2]                         # each rank its own batch


def test_reference_arm_runs_on_rank0_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference"])
    bench.run_reference(bench._args())
    assert capsys.readouterr().out == ""                  # no work, no line on rank 1
