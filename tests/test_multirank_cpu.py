"""Replica scaling of the benchmark (independent jobs per rank, no data-path
collective): two gloo ranks on CPU check that the reported time is the
slowest rank's and that the whole-job rate counts every rank's job."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [400.0, 650.0][rank]
    ms = bench.max_over_ranks(ms_local, dist, torch.device("cpu"))
    out[rank] = (ms, bench.whole_job_rate(world, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_count_all_jobs():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, rate = out[r]
        assert ms == 650.0
        assert abs(rate - 2 * 1e3 / 650.0) < 1e-12


def test_single_rank_is_the_local_time():
    import bench
    assert bench.max_over_ranks(123.0, None, None) == 123.0
    assert bench.whole_job_rate(1, 500.0) == 2.0
