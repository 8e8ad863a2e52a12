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
    ``elem`` per row) into the full vector, ``reduce`` adds the ranks' sums.
    With ``host=True`` (a process group whose backend takes CPU tensors, such
    as gloo) both go through host memory."""

    def __init__(self, bounds, elem: int, group=None, host: bool = False):
        self.bounds = [(int(a), int(b)) for a, b in bounds]
        self.elem = int(elem)
        self.group = group
        self.host = bool(host)
        self.longest = max(b - a for a, b in self.bounds) * self.elem

    def gather(self, w):
        import torch
        import torch.distributed as dist
        rank = dist.get_rank(self.group)
        e, L = self.elem, self.longest
        a, b = self.bounds[rank]
        dev = torch.device("cpu") if self.host else w.device
        send = torch.zeros(L, dtype=torch.uint8, device=dev)
        send[:(b - a) * e] = w[a * e:b * e].to(dev)
        recv = torch.empty(len(self.bounds) * L, dtype=torch.uint8, device=dev)
        dist.all_gather(list(recv.split(L)), send, group=self.group)
        for r, (a, b) in enumerate(self.bounds):
            if r != rank:
                w[a * e:b * e].copy_(recv[r * L:r * L + (b - a) * e])

    def reduce(self, sums):
        import torch.distributed as dist
        if self.host:
            h = sums.cpu()
            dist.all_reduce(h, group=self.group)
            sums.copy_(h)
        else:
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

    def run(self, kind: int, sums, ctl, w_in=None, w_out=None, ranks=None, damping: float = 0.0,
            tol: float = 0.0, max_iter: int = 1, stream=None):
        import paper_2210_01465_gb300 as ffg
        op = ffg.ffg_rows_op(int(kind), int(max_iter), float(damping), float(tol),
                             None if w_in is None else w_in.data_ptr(),
                             None if w_out is None else w_out.data_ptr(),
                             None if ranks is None else ranks.data_ptr(), sums.data_ptr(),
                             ctl.data_ptr())
        ffg._check(ffg.pagerank_rows_run(self.g.c, self.row0, self.row1, self.prec, op,
                                         self.ws.data_ptr(), self.need,
                                         ffg._stream_handle(stream)),
                   "pagerank_rows_run")


def solve_rows(g, ranges, damping: float = 0.85, tol: float = 1e-12, max_iter: int = 10000,
               prec=None, exchange=None, init=None, stream=None):
    """Row-partitioned PageRank of ``g``: this process works on ``ranges``
    ((row0, row1) pairs, or RowRange objects laid out before).  Several
    ranges in one process stand for several ranks (their rows of w land in
    the same buffers, nothing to exchange); between processes ``exchange``
    (a RowExchange) all-gathers w and adds the sums, and the ranges of all
    ranks must cover every row.  Every decision -- the stopping rule, the
    teleport term, the normalisation -- is taken on the device from the
    summed fixed-point values (pagerank_rows_run's control operations), with
    pagerank_solve's arithmetic, so FP64 results equal its bit for bit; this
    function only moves bytes and reads the stop flag once per iteration.
    Returns (ranks, iterations, residual, converged); the ranks hold every
    row after an exchange, else this process's rows."""
    import numpy as np
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
    ctl = torch.zeros(ffg.ROWS_CTL_BYTES, dtype=torch.uint8, device=dev)
    dt = torch.float64 if prec == ffg.F64 else torch.float32
    ranks = torch.zeros(n, dtype=dt, device=dev)
    head = parts[0]   # the control operations run once per process

    def flags():
        c = ctl[:16].cpu().numpy().view(np.int32)   # iters, stop, converged, status
        if c[3]:
            raise ffg.FFGError(int(c[3]), "pagerank_rows_run")
        return c

    for p in parts:
        p.run(ffg.ROWS_INIT, sums, ctl, w_out=w_cur, ranks=init, stream=stream)
    if exchange is not None:
        exchange(w_cur, sums)
    head.run(ffg.ROWS_START, sums, ctl, stream=stream)
    while True:
        for p in parts:
            p.run(ffg.ROWS_STEP, sums, ctl, w_in=w_cur, w_out=w_next, damping=damping,
                  stream=stream)
        if exchange is not None:
            exchange(w_next, sums)
        head.run(ffg.ROWS_ADVANCE, sums, ctl, tol=tol, max_iter=max_iter, stream=stream)
        w_cur, w_next = w_next, w_cur
        if flags()[1]:
            break
    for p in parts:
        p.run(ffg.ROWS_SUM, sums, ctl, w_in=w_cur, stream=stream)
    if exchange is not None:
        exchange.reduce(sums)
    head.run(ffg.ROWS_SCALE, sums, ctl, stream=stream)
    for p in parts:
        p.run(ffg.ROWS_WRITE, sums, ctl, w_in=w_cur, ranks=ranks, stream=stream)
    if exchange is not None:
        # every row's ranks on every rank: gather them like w
        raw = ranks.view(torch.uint8)
        RowExchange(exchange.bounds, ranks.element_size(), exchange.group,
                    exchange.host).gather(raw)
    c = ctl.cpu().numpy()
    it, _, conv, _ = c[:16].view(np.int32)
    res = float(c[16:24].view(np.float64)[0])
    return ranks, int(it), res, bool(conv)
