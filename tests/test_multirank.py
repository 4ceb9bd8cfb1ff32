"""Multi-rank host logic of bench.py (replicas, max-over-ranks timing) with
two gloo ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    ms = 10.0 + 5.0 * rank            # rank 1 is the slow replica
    m = bench.max_over_ranks(ms, dist, "cpu")
    dist.barrier()
    out[rank] = m
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 15.0


def test_job_throughput_counts_all_replicas():
    import bench
    v1 = bench.job_throughput(1, 1000, 10, 2.0)
    v2 = bench.job_throughput(2, 1000, 10, 2.0)
    assert abs(v2 - 2 * v1) < 1e-12 and abs(v1 - 1000 * 10 / 2e-3 / 1e6) < 1e-12
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
