"""The replicas-only multi-GPU path of bench.py, on CPU with gloo (world size 2)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, results):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r: 4 roots of m = 1e9 tuples, each taking (r + 1) ms
    t = [(rank + 1) * 1e-3] * 4
    m = [10 ** 9] * 4
    inv = sum(ti / mi for ti, mi in zip(t, m))
    value, ms = bench.job_value(inv, 1e3 * sum(t), 4, dist, torch.device("cpu"))
    results[rank] = (value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_job_value_is_the_slowest_rank_over_all_roots():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    results = manager.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, results), nprocs=2, join=True, start_method="spawn")
    # slowest rank: 4 roots at 2 ms each -> sum t/m = 8e-12; 8 roots / 8e-12 = 1e12 TEPS = 1000 GTEPS
    for rank in (0, 1):
        value, ms = results[rank]
        assert value == pytest.approx(1000.0)
        assert ms == pytest.approx(8.0)


def test_job_value_single_process():
    import bench
    value, ms = bench.job_value(4e-12, 4.0, 4)
    assert value == pytest.approx(1000.0) and ms == 4.0
