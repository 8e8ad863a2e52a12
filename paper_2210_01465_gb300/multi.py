"""Several GPUs: the spaces of a batch are independent, so they are sharded
across ranks with no collective on the data path; only the timings and
counts are reduced at the end (max of times, sum of work)."""
from __future__ import annotations

import heapq


def shard_lpt(costs, world: int):
    """Longest-processing-time-first assignment of jobs to ``world`` ranks.
    Returns a list of job-index lists, one per rank (deterministic)."""
    order = sorted(range(len(costs)), key=lambda j: (-costs[j], j))
    heap = [(0.0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for j in order:
        load, r = heapq.heappop(heap)
        out[r].append(j)
        heapq.heappush(heap, (load + costs[j], r))
    return [sorted(x) for x in out]


def reduce_time_work(ms: float, units: float, group=None, device="cpu"):
    """(max over ranks of ms, sum over ranks of units) through torch.distributed."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return ms, units
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), float(u.item())


# ---------------------------------------------------------------------------
# one graph over several ranks: the row-partitioned PageRank (rows split by
# cost, w exchanged by an all-gather and the sums by an all-reduce between
# iterations)
# ---------------------------------------------------------------------------

FIX = float(1 << 60)  # quantum of the fixed-point sums: 2^-60


def split_rows(in_ptr, parts: int, row_cost: int = 20):
    """Contiguous row ranges [(row0, row1), ...] covering every row, of about
    equal cost (in-edges + ``row_cost`` per row).  ``in_ptr``: host array of
    n + 1 row pointers."""
    import numpy as np
    ptr = np.asarray(in_ptr, dtype=np.int64)
    n = len(ptr) - 1
    if parts < 1 or n < parts:
        raise ValueError(f"cannot split {n} rows into {parts} ranges")
    cost = ptr - ptr[0] + row_cost * np.arange(n + 1, dtype=np.int64)
    cuts = [0]
    for k in range(1, parts):
        c = int(np.searchsorted(cost, cost[-1] * k / parts))
        cuts.append(min(max(c, cuts[-1] + 1), n - (parts - k)))
    cuts.append(n)
    return list(zip(cuts[:-1], cuts[1:]))


class RowExchange:
    """The exchange of a row-partitioned solve between processes: rank r owns
    ``bounds[r]``; ``gather`` all-gathers every rank's rows of w (bytes,
    ``elem`` per row) into the full vector, ``reduce`` adds the ranks' sums."""

    def __init__(self, bounds, elem: int, group=None):
        self.bounds = [(int(a), int(b)) for a, b in bounds]
        self.elem = int(elem)
        self.group = group
        self.longest = max(b - a for a, b in self.bounds) * self.elem

    def gather(self, w):
        import torch
        import torch.distributed as dist
        rank = dist.get_rank(self.group)
        e, L = self.elem, self.longest
        a, b = self.bounds[rank]
        send = torch.zeros(L, dtype=torch.uint8, device=w.device)
        send[:(b - a) * e] = w[a * e:b * e]
        parts = [torch.empty(L, dtype=torch.uint8, device=w.device) for _ in self.bounds]
        dist.all_gather(parts, send, group=self.group)
        for (a, b), p in zip(self.bounds, parts):
            w[a * e:b * e] = p[:(b - a) * e]

    def reduce(self, sums):
        import torch.distributed as dist
        dist.all_reduce(sums, group=self.group)

    def __call__(self, w, sums):
        self.gather(w)
        self.reduce(sums)


class RowRange:
    """Rows [row0, row1) of a graph, laid out for ``pagerank_rows_run``."""

    def __init__(self, g, row0: int, row1: int, prec: int, stream=None):
        import paper_2210_01465_gb300 as ffg
        self.g, self.row0, self.row1, self.prec = g, int(row0), int(row1), prec
        need = ffg.pagerank_rows_workspace_bytes(g.c, self.row0, self.row1, prec)
        if need == 0:
            raise ffg.FFGError(ffg.FFG_ERR_INVALID_ARG, "pagerank_rows_workspace_bytes: " +
                               ffg.ffg_last_error())
        self.need = need
        self.ws = ffg.workspace(need, g.out_ptr.device)
        ffg._check(ffg.pagerank_rows_prepare(g.c, self.row0, self.row1, prec, self.ws.data_ptr(),
                                             need, ffg._stream_handle(stream)),
                   "pagerank_rows_prepare")

    def run(self, kind: int, sums, w_in=None, w_out=None, ranks=None, damping: float = 0.0,
            dangling: int = 0, scale: float = 1.0, stream=None):
        import paper_2210_01465_gb300 as ffg
        op = ffg.ffg_rows_op(int(kind), 0, float(damping), int(dangling), float(scale),
                             None if w_in is None else w_in.data_ptr(),
                             None if w_out is None else w_out.data_ptr(),
                             None if ranks is None else ranks.data_ptr(), sums.data_ptr())
        ffg._check(ffg.pagerank_rows_run(self.g.c, self.row0, self.row1, self.prec, op,
                                         self.ws.data_ptr(), self.need,
                                         ffg._stream_handle(stream)),
                   "pagerank_rows_run")


def solve_rows(g, ranges, damping: float = 0.85, tol: float = 1e-12, max_iter: int = 10000,
               prec=None, exchange=None, init=None, stream=None):
    """Row-partitioned PageRank of ``g``: this process works on ``ranges``
    ((row0, row1) pairs, or RowRange objects laid out before).  Several ranges in one process stand for several
    ranks (their rows of w land in the same buffers, nothing to exchange);
    between processes ``exchange`` (a RowExchange) all-gathers w and adds
    the sums, and the ranges of all ranks must cover every row.  The stopping
    rule and the normalisation are pagerank_solve's, so FP64 results equal
    its bit for bit.  Returns (ranks, iterations, residual, converged); the
    ranks hold every row after an exchange, else this process's rows."""
    import torch
    import paper_2210_01465_gb300 as ffg
    prec = ffg.F64 if prec is None else prec
    dev = g.out_ptr.device
    n = g.n_nodes
    wb = ffg.pagerank_rows_w_bytes(prec)
    parts = [r if isinstance(r, RowRange) else RowRange(g, r[0], r[1], prec, stream)
             for r in ranges]
    w_cur = torch.zeros(n * wb, dtype=torch.uint8, device=dev)
    w_next = torch.zeros(n * wb, dtype=torch.uint8, device=dev)
    sums = torch.zeros(4, dtype=torch.int64, device=dev)
    dt = torch.float64 if prec == ffg.F64 else torch.float32
    ranks = torch.zeros(n, dtype=dt, device=dev)

    def settle(w):
        if exchange is not None:
            exchange(w, sums)
        s = [int(v) for v in sums.cpu()]
        if s[3]:
            raise ffg.FFGError(ffg.FFG_ERR_TIMEOUT, "pagerank_rows_run")
        return s

    for p in parts:
        p.run(ffg.ROWS_INIT, sums, w_out=w_cur, ranks=init, stream=stream)
    dangling = settle(w_cur)[1]
    it, res, converged = 0, float("inf"), False
    while True:
        sums.zero_()
        for p in parts:
            p.run(ffg.ROWS_STEP, sums, w_in=w_cur, w_out=w_next, damping=damping,
                  dangling=dangling, stream=stream)
        s = settle(w_next)
        prev, res, dangling = res, s[0] / FIX, s[1]
        it += 1
        w_cur, w_next = w_next, w_cur
        if res < tol or (prec == ffg.F32 and res >= prev):
            converged = True
            break
        if it >= max_iter:
            break
    sums.zero_()
    for p in parts:
        p.run(ffg.ROWS_SUM, sums, w_in=w_cur, stream=stream)
    if exchange is not None:
        exchange.reduce(sums)
    xs = int(sums.cpu()[2]) / FIX
    for p in parts:
        p.run(ffg.ROWS_WRITE, sums, w_in=w_cur, ranks=ranks, scale=1.0 / xs, stream=stream)
    if exchange is not None:
        # every row's ranks on every rank: gather them like w
        raw = ranks.view(torch.uint8)
        RowExchange(exchange.bounds, ranks.element_size(), exchange.group).gather(raw)
    return ranks, it, res, converged
