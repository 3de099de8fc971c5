"""bench.py's whole-job aggregation across ranks, with two gloo ranks on CPU.

Each rank reconstructs its own volumes (replicas: the path has no exchange
step), so the job's time per step is the slowest rank's and the throughput is
all ranks' voxels over that time."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [2.0, 3.0][rank]
    ms, value = bench.aggregate(local_ms, 1024 * 1024 * 256, world, dist)
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregate_takes_slowest_rank():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    expect = 2 * 1024 * 1024 * 256 / 3.0e-3 / 1e9
    for r in range(2):
        ms, value = out[r]
        assert ms == 3.0
        assert abs(value - expect) < 1e-9 * expect


def test_single_rank_aggregate_is_local():
    import bench
    ms, value = bench.aggregate(2.5, 1000, 1)
    assert ms == 2.5 and abs(value - 1000 / 2.5e-3 / 1e9) < 1e-15
