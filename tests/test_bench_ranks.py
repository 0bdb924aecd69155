"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own
step time; the job time is the slowest rank's and the throughput counts the
builds of every rank (weak scaling, no collective on the data path)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    my_ms = 100.0 + 50.0 * rank          # rank 1 is the slowest
    job_ms = bench.max_over_ranks(my_ms, dist, "cpu")
    out[rank] = (job_ms, bench.job_throughput(world, 20, job_ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        job_ms, value = out[r]
        assert job_ms == 150.0
        assert value == pytest.approx(2 * 20 / 0.150)


def test_single_rank_is_identity():
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.job_throughput(1, 10, 1000.0) == pytest.approx(10.0)
