"""Multi-rank host logic on CPU: two gloo ranks shard regions, reduce the timing, and
agree on the whole-job throughput (no GPU, no data-path collective)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1604_02292_gb300 import shard
from paper_1604_02292_gb300 import workloads as WL


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = WL.BATCHES["roi_batch_2048"]
        items = WL.batch_regions(w, seed=0, count=64)
        costs = [shard.region_cost(r, p["iters"], w.n_angles) for r, p in items]
        mine = shard.assign(costs, world)[rank]
        # every rank computes the same assignment; gather to check disjointness
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        fake_seconds = 1.0 + rank          # rank 1 is slower
        tmax = shard.max_over_ranks(fake_seconds, dist)
        value = shard.throughput(10, world, tmax)
        q.put((rank, gathered, tmax, value, sum(costs[i] for i in mine), sum(costs)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    g0, g1 = res[0][1], res[1][1]
    assert g0 == g1
    allidx = sorted(g0[0] + g0[1])
    assert allidx == list(range(64)) and not set(g0[0]) & set(g0[1])
    for rank, _, tmax, value, mine, total in res:
        assert tmax == 2.0 and value == pytest.approx(10 * 2 / 2.0)
        assert abs(mine - total / 2) <= 0.1 * total   # balanced to within 10 %


def test_assign_is_lpt_and_deterministic():
    costs = [5.0, 3.0, 3.0, 2.0, 2.0, 2.0]
    a = shard.assign(costs, 2)
    assert a == shard.assign(costs, 2)
    loads = [sum(costs[i] for i in s) for s in a]
    assert sorted(loads) == [8.0, 9.0]
    assert shard.assign(costs, 1) == [list(range(6))]
    with pytest.raises(ValueError):
        shard.assign(costs, 0)
