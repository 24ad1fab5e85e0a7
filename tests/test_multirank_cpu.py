"""Host logic of the multi-GPU paths, run as 2 gloo ranks on the CPU: the batch shard
assignment covers every matrix exactly once and balances the cost, and the timing
reduction takes the maximum over ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth

    specs = synth.batch_specs(64, rows_lo=100, rows_hi=5000)
    costs = [sp.rows * (5 if sp.kind == "stencil2d" else sp.avg) for sp in specs]
    mine = bench.shard_for_rank(costs, world, rank)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        q.put((gathered, costs, float(t[0])))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_batch_sharding_two_gloo_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered, costs, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    flat = sorted(i for part in gathered for i in part)
    assert flat == list(range(len(costs)))  # every matrix exactly once
    loads = [sum(costs[i] for i in part) for part in gathered]
    assert max(loads) <= 1.1 * sum(loads) / world + max(costs)  # greedy LPT bound
    assert tmax == float(world)
