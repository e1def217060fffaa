"""The multi-rank host logic of bench.py on CPU with gloo: replicas report
the slowest rank's time and the units of all ranks (bench.aggregate, which
every leg of the bench goes through), and the batched sweep's 48 instances
are split across ranks without overlap, also when the shards hold different
numbers of points (5 ranks)."""
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
    import workloads as W

    def rmax(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def rsum(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())

    local_ms = 100.0 + 150.0 * rank                    # the last rank is the slowest
    local_units = 4.0e6 * (rank + 1)
    replicas = bench.aggregate(local_ms, local_units, world, rmax, rsum)
    # the sweep leg: this rank's shard of the real instance list, its points per step
    mine = bench.shard(48, rank, world)
    pts = float(sum(W.sweep_instance(i).npts for i in mine))
    sweep = bench.aggregate(10.0 + rank, pts * 5, world, rmax, rsum)
    got = [None] * world
    dist.all_gather_object(got, (mine, pts))
    dist.barrier()
    if rank == 0:
        q.put((replicas, sweep, got))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 5])
def test_replica_aggregation_and_sweep_sharding_gloo(world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    (ms, units, rate), (sms, sunits, srate), got = q.get(timeout=10)
    assert ms == 100.0 + 150.0 * (world - 1)
    assert units == sum(4.0e6 * (r + 1) for r in range(world))
    assert rate == pytest.approx(units / (ms / 1e3))
    shards = [g[0] for g in got]
    flat = sorted(i for s in shards for i in s)
    assert flat == list(range(48))
    assert all(not set(a) & set(b) for k, a in enumerate(shards) for b in shards[k + 1:])
    # 16 each of 128^2, 256^2, 512^2: the whole job's points whatever the split
    total = 16 * (128 ** 2 + 256 ** 2 + 512 ** 2)
    assert sum(g[1] for g in got) == total
    assert sunits == total * 5 and sms == 10.0 + (world - 1)
    assert srate == pytest.approx(total * 5 / (sms / 1e3))
    if world == 5:  # uneven shards: the points differ from rank to rank
        assert len({g[1] for g in got}) > 1
