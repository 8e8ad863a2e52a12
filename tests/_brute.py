"""Brute-force definitions used to pin the oracle (pure Python / numpy).

These restate the paper's definitions in the least clever way available and
are independent of both the oracle and the CUDA library:

* points of X = S_1 x ... x S_n in itertools.product order (Sec. III-B),
* clause evaluation with Python's unbounded integers,
* neighbours by an all-pairs scan for Hamming distance one (Eq. 2) or for one
  coordinate that moves by one list position (adjacent, Sec. III-B),
* the FFG edge rule "neighbour with lower fitness" (Sec. VII-B),
* PageRank as the solution of the dense Google linear system.
"""
import itertools
import math

import numpy as np


def clause_holds(vals, cl):
    pa = math.prod(vals[i] for i in cl.a)
    pb = math.prod(vals[i] for i in cl.b)
    if cl.kind == "prod_le":
        return pa <= cl.bound
    if cl.kind == "prod_ge":
        return pa >= cl.bound
    if cl.kind == "divides":
        return pb != 0 and pa % pb == 0
    if cl.kind == "prod_le_prod":
        return pa <= pb
    raise ValueError(cl.kind)


def positions(spec):
    """All list-position tuples in row-major order (last parameter fastest)."""
    return list(itertools.product(*[range(len(v)) for v in spec.values]))


def valid_mask(spec):
    out = []
    for pos in positions(spec):
        vals = [spec.values[i][p] for i, p in enumerate(pos)]
        out.append(all(clause_holds(vals, cl) for cl in spec.clauses))
    return np.array(out, dtype=bool)


def keys(fitness, fail_thr=1e10):
    f = np.asarray(fitness, dtype=np.float64)
    failed = ~(f < fail_thr)
    return np.where(failed, np.inf, f), failed


def edge_lists(spec, fitness_raw, nbh="hamming", fail_thr=1e10):
    """(node_raw, out_lists, in_lists, failed) of the FFG by brute force."""
    valid = valid_mask(spec)
    node_raw = np.flatnonzero(valid)
    P = np.array(positions(spec), dtype=np.int64)[node_raw]
    key, failed = keys(np.asarray(fitness_raw)[node_raw], fail_thr)
    N = len(node_raw)
    out_lists = [[] for _ in range(N)]
    for u in range(N):
        d = P - P[u]
        ndiff = (d != 0).sum(axis=1)
        if nbh == "hamming":
            nb = np.flatnonzero(ndiff == 1)
        else:
            nb = np.flatnonzero((ndiff == 1) & (np.abs(d).sum(axis=1) == 1))
        out_lists[u] = sorted(int(v) for v in nb if key[v] < key[u])
    in_lists = [[] for _ in range(N)]
    for u in range(N):
        for v in out_lists[u]:
            in_lists[v].append(u)
    return node_raw, out_lists, [sorted(x) for x in in_lists], failed


def neighbour_count(spec, nbh="hamming"):
    """Number of valid neighbours of every valid point."""
    valid = valid_mask(spec)
    node_raw = np.flatnonzero(valid)
    P = np.array(positions(spec), dtype=np.int64)[node_raw]
    out = np.zeros(len(node_raw), dtype=np.int64)
    for u in range(len(node_raw)):
        d = P - P[u]
        ndiff = (d != 0).sum(axis=1)
        if nbh == "hamming":
            out[u] = int((ndiff == 1).sum())
        else:
            out[u] = int(((ndiff == 1) & (np.abs(d).sum(axis=1) == 1)).sum())
    return out


def dense_pagerank(out_lists, alpha):
    """Solve (I - alpha P - alpha/N 1 d^T) x = (1-alpha)/N 1 with numpy.

    P[v,u] = 1/outdeg(u) for every edge u->v (each column of the adjacency
    matrix rescaled to sum to one), d = indicator of nodes without out-edges.
    """
    N = len(out_lists)
    A = np.eye(N)
    for u, outs in enumerate(out_lists):
        if outs:
            for v in outs:
                A[v, u] -= alpha / len(outs)
        else:
            A[:, u] -= alpha / N
    b = np.full(N, (1.0 - alpha) / N)
    return np.linalg.solve(A, b)


def csr(lists):
    ptr = np.zeros(len(lists) + 1, dtype=np.int64)
    ptr[1:] = np.cumsum([len(x) for x in lists])
    idx = np.array([v for x in lists for v in x], dtype=np.int32)
    return ptr, idx
