"""The multi-rank host logic of bench.py on CPU with gloo, world_size 2:
replicas report the slowest rank's time and the units of all ranks, and the
batched sweep's instances are split across ranks without overlap."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    def rmax(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def rsum(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())

    local_ms = 100.0 if rank == 0 else 250.0          # rank 1 is the slow one
    local_units = 4.0e6 * (rank + 1)
    ms, units, rate = bench.aggregate(local_ms, local_units, world, rmax, rsum)
    mine = bench.shard(48, rank, world)
    got = [None] * world
    dist.all_gather_object(got, mine)
    dist.barrier()
    if rank == 0:
        q.put((ms, units, rate, got))
    dist.destroy_process_group()


def test_replica_aggregation_and_sweep_sharding_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    ms, units, rate, shards = q.get(timeout=10)
    assert ms == 250.0
    assert units == 4.0e6 + 8.0e6
    assert rate == pytest.approx(12.0e6 / 0.25)
    flat = sorted(i for s in shards for i in s)
    assert flat == list(range(48))
    assert not set(shards[0]) & set(shards[1])
