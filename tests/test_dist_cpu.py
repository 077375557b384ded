"""The N > 1 path of bench.py (one replica per rank) on CPU with the gloo
backend and world size 2: the barrier, the max-over-ranks timing and the
whole-job rate, and the reference arm's rank-0-only rule."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = bench.dist_env()
        bench.barrier(w)
        mx = bench.max_over_ranks(times[r], w)
        out[r] = (r, w, mx, bench.whole_job_rate(1000.0, mx, w))
        bench.barrier(w)
    finally:
        dist.destroy_process_group()


def test_replicas_max_over_ranks_and_rate():
    world, port = 2, _free_port()
    times = [0.5, 0.8]
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, port, times, out), nprocs=world, start_method="spawn")
        res = dict(out)
    assert set(res) == {0, 1}
    for r in (0, 1):
        rank, w, mx, rate = res[r]
        assert rank == r and w == 2
        assert mx == pytest.approx(0.8)                  # every rank sees the slowest rank's time
        assert rate == pytest.approx(2 * 1000.0 / 0.8)   # all replicas' units over that time


def test_reference_arm_runs_on_rank0_only(monkeypatch, capsys):
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    calls = []
    monkeypatch.setattr(bench, "cpu_baseline", lambda *a, **k: calls.append(1))
    bench.run_reference(argparse.Namespace(config="cfg1", steps=2, warmup=3))
    assert calls == [] and capsys.readouterr().out == ""
