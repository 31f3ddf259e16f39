"""The multi-GPU form of the benchmark is independent replicas (the path has
no exchange step between structures): each rank times its own steps, the
job's time is the slowest rank's, and the throughput counts every rank's
atom-steps.  This checks that aggregation over two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ms_by_rank, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(ms_by_rank[rank], dist, device="cpu")
        out[rank] = (ms, bench.job_throughput(world, 1_000_000, 10, ms))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    ms_by_rank = [120.0, 150.0]
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, _free_port(), ms_by_rank, out), nprocs=world, start_method="spawn")
        res = dict(out)
    assert res[0] == res[1]
    ms, value = res[0]
    assert ms == 150.0
    # 2 replicas x 1e6 atoms x 10 steps in 0.15 s
    assert abs(value - 2 * 1e6 * 10 / 0.15 / 1e6) < 1e-9


def test_single_process_is_identity():
    assert bench.max_over_ranks(42.0) == 42.0
    assert bench.job_throughput(1, 2_000_000, 5, 1000.0) == 10.0
