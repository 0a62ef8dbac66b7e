"""Host-side logic of the multi-GPU benchmark, on CPU with two gloo ranks:
replicas or batched samples are sharded with no data-path collective; only
the timing is reduced (max over ranks)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


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
    costs = [50000, 5000, 32000, 17000, 44000, 9000, 21000]
    shards = bench.shard_samples(costs, world)
    mine = shards[rank]
    units = float(sum(costs[i] for i in mine))
    elapsed = 1.0 + 0.5 * rank  # pretend rank 1 is slower
    t = torch.tensor([elapsed])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([units])
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    q.put((rank, mine, float(t.item()), float(u.item())))
    dist.destroy_process_group()


def test_two_rank_sharding_and_timing():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shards = [r[1] for r in res]
    costs = [50000, 5000, 32000, 17000, 44000, 9000, 21000]
    # every sample exactly once, loads balanced within the largest sample
    assert sorted(i for s in shards for i in s) == list(range(len(costs)))
    loads = [sum(costs[i] for i in s) for s in shards]
    assert abs(loads[0] - loads[1]) <= max(costs)
    # both ranks agree on the slowest time and the total units
    assert res[0][2] == res[1][2] == 1.5
    assert res[0][3] == res[1][3] == float(sum(costs))
    assert bench.aggregate(loads, [1.0, 1.5]) == pytest.approx(sum(costs) / 1.5)
