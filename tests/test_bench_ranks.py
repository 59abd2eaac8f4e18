"""The multi-process path of bench.py on CPU (gloo, two ranks): every rank
gets the slowest rank's time, the job's rate counts the units of all ranks,
and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, times, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(times[rank], dist, "cpu")
        out[rank] = (ms, bench.job_rate(3, world, ms))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_with_two_gloo_ranks():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    times = [120.0, 200.0]
    mp.start_processes(_rank, args=(2, _free_port(), times, out), nprocs=2, join=True, start_method="spawn")
    assert dict(out) == {0: (200.0, 3 * 2 / 0.2), 1: (200.0, 3 * 2 / 0.2)}


def test_single_process_is_its_own_max():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    assert bench.job_rate(10, 1, 500.0) == 20.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(workload="c4", warmup=0, steps=1, gpus=2)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
