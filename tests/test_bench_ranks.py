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


def _shard_rank(rank, world, port, out):
    """One rank of a g-sharded build: the oracle's share of its slice (V and W
    rows outside the slice set to zero: every line of Eq. exoccri is a sum
    over the rows g), then bench.reduce_partials over gloo."""
    import numpy as np
    import torch
    import oracle
    from cellgen import build_cell, config_spec
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    c = build_cell(config_spec(1))
    g0, g1 = bench.shard_slices(c.idx.size, world)[rank]
    Vs = np.zeros_like(c.V)
    Ws = np.zeros_like(c.W)
    Vs[g0:g1] = c.V[g0:g1]
    Ws[g0:g1] = c.W[g0:g1]
    Kp, Ep = oracle.exx_rps_occri(c.phi, c.idx, Vs, Ws, c.C, c.dV)
    K = torch.from_numpy(np.ascontiguousarray(Kp))
    E = torch.tensor([Ep], dtype=torch.float64)
    bench.reduce_partials(K, E, dist)
    out[rank] = (K.numpy().copy(), float(E.item()))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_partials_reduce_to_the_full_build():
    """The g-sharded decomposition on CPU: two gloo ranks each hold one slice
    of the interpolation points; their shares of K_{mu i} and E_x, summed by
    the bench's single allreduce, equal the unsharded oracle build."""
    import numpy as np
    import oracle
    from cellgen import build_cell, config_spec
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_shard_rank, args=(world, port, out), nprocs=world, join=True)
    c = build_cell(config_spec(1))
    K0, E0 = oracle.exx_rps_occri(c.phi, c.idx, c.V, c.W, c.C, c.dV)
    assert bench.shard_slices(256, 2) == [(0, 128), (128, 256)]
    for r in range(world):
        K, E = out[r]
        assert np.max(np.abs(K - K0)) <= 1e-12 * np.max(np.abs(K0))
        assert abs(E - E0) <= 1e-12 * abs(E0)


def test_single_rank_is_identity():
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.job_throughput(1, 10, 1000.0) == pytest.approx(10.0)


def test_reference_arm_json_line():
    """`bench.py --impl reference` (the oracle on the host) prints one JSON
    line with the keys the benchmark contract asks for."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--config", "1", "--steps", "1", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle"
