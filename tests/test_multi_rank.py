"""Multi-rank host logic on CPU with the gloo backend (world size 2)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2210_01465_gb300.multi import reduce_time_work, shard_lpt


def test_shard_lpt_covers_and_balances():
    costs = [float(c) for c in [5, 9, 1, 1, 7, 3, 3, 8, 2, 2, 6]]
    for world in (1, 2, 3, 4):
        parts = shard_lpt(costs, world)
        flat = sorted(j for p in parts for j in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[j] for j in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs)
    assert shard_lpt(costs, 2) == shard_lpt(list(costs), 2)  # deterministic


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    costs = [float(10 + (7 * k) % 13) for k in range(40)]
    mine = shard_lpt(costs, world)[rank]
    work = sum(costs[j] for j in mine)
    ms = 100.0 + 10.0 * rank
    t, u = reduce_time_work(ms, work)
    import torch
    got = [None] * world
    dist.all_gather_object(got, mine)
    dist.destroy_process_group()
    q.put((rank, t, u, got))


@pytest.mark.timeout(120)
def test_two_ranks_gloo_reduce_and_disjoint_shards():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=100) for _ in range(world)]
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    costs = [float(10 + (7 * k) % 13) for k in range(40)]
    for rank, t, u, got in res:
        assert t == 110.0                       # max over ranks
        assert abs(u - sum(costs)) < 1e-9       # all work counted once
        assert sorted(got[0] + got[1]) == list(range(40))
        assert not set(got[0]) & set(got[1])
