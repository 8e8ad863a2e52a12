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


# ------------------------------------------------- one graph split by rows

def test_split_rows_covers_and_balances():
    import numpy as np
    from paper_2210_01465_gb300.multi import split_rows
    rng = np.random.default_rng(5)
    deg = rng.integers(0, 60, size=1000)
    in_ptr = np.concatenate([[0], np.cumsum(deg)])
    for parts in (1, 2, 3, 7, 16):
        b = split_rows(in_ptr, parts)
        assert b[0][0] == 0 and b[-1][1] == 1000 and len(b) == parts
        assert all(r0 < r1 for r0, r1 in b)
        assert all(b[k][1] == b[k + 1][0] for k in range(parts - 1))
        cost = [int(in_ptr[r1] - in_ptr[r0]) + 20 * (r1 - r0) for r0, r1 in b]
        assert max(cost) - min(cost) <= 2 * (deg.max() + 20)
    assert split_rows([0, 1, 2, 3], 3) == [(0, 1), (1, 2), (2, 3)]
    with pytest.raises(ValueError):
        split_rows([0, 1, 2], 3)


def _rows_worker(rank, world, port, q):
    """A row-partitioned power iteration on a small FFG: every rank updates
    its rows (numpy stands in for the device step), then RowExchange shares
    w and adds the fixed-point sums."""
    import numpy as np
    import torch
    import torch.distributed as dist
    import ffg_inputs as fi
    import oracle
    from paper_2210_01465_gb300.multi import FIX, RowExchange, split_rows
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    spec = fi.single_small()
    og = oracle.build(spec, fi.runtimes(spec, 3), oracle.HAMMING)
    n, alpha = og.n_nodes, 0.85
    bounds = split_rows(og.in_ptr, world)
    r0, r1 = bounds[rank]
    ex = RowExchange(bounds, 8)
    od = og.outdeg
    w = torch.zeros(n, dtype=torch.float64)
    x0 = 1.0 / n
    w[r0:r1] = torch.from_numpy(np.where(od[r0:r1] > 0, x0 / np.maximum(od[r0:r1], 1), x0))
    sums = torch.zeros(4, dtype=torch.int64)
    sums[1] = int(round(x0 * (od[r0:r1] == 0).sum() * FIX))
    ex(w.view(torch.uint8), sums)
    dangling = int(sums[1]) / FIX
    for it in range(60):
        wn = w.clone()
        c = (alpha * dangling + 1.0 - alpha) / n
        xs_new = np.empty(r1 - r0)
        for v in range(r0, r1):
            s = sum(float(w[u]) for u in og.in_idx[og.in_ptr[v]:og.in_ptr[v + 1]])
            xs_new[v - r0] = alpha * s + c
        wn[r0:r1] = torch.from_numpy(np.where(od[r0:r1] > 0, xs_new / np.maximum(od[r0:r1], 1),
                                              xs_new))
        sums.zero_()
        sums[1] = int(round(float(xs_new[od[r0:r1] == 0].sum()) * FIX))
        ex(wn.view(torch.uint8), sums)
        dangling = int(sums[1]) / FIX
        w = wn
    x = np.where(od > 0, w.numpy() * od, w.numpy())
    dist.destroy_process_group()
    q.put((rank, x))


@pytest.mark.timeout(240)
@pytest.mark.parametrize("world", [2, 3])
def test_gloo_row_exchange_power_iteration(world):
    import numpy as np
    import ffg_inputs as fi
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rows_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=150) for _ in range(world))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    spec = fi.single_small()
    og = oracle.build(spec, fi.runtimes(spec, 3), oracle.HAMMING)
    xo, _, _, _ = oracle.pagerank_power(og, 0.85, 0.0, max_iter=60)
    for rank in range(world):   # every rank holds every row, equal to the oracle's iterate
        assert np.abs(res[rank] - xo).sum() < 1e-12
        np.testing.assert_array_equal(res[rank], res[0])
