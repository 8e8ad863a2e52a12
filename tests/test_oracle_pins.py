"""Pins of the CPU oracle against the paper and against mathematics.

Each test checks the oracle against something that is not the oracle: the
paper's printed numbers and worked example, brute-force restatements of the
definitions, a dense linear solve, closed forms, a library routine, or
invariants.  None of these tests needs a GPU.
"""
import math
import os

import numpy as np
import pytest

import ffg_inputs as fi
import oracle
from ffg_inputs import Clause, SpaceSpec

from . import _brute as brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _one_param(values, clauses=()):
    return SpaceSpec("one", ("p",), (tuple(values),), tuple(clauses))


# ---------------------------------------------------------------- search space

def test_paper_space_sizes():
    """Sec. V table: #points of each kernel space = product of its list lengths."""
    for name, count in _read_golden("paper_space_sizes.txt"):
        make, _ = fi.PAPER_SPACES[name]
        assert oracle.raw_count(make()) == int(count), name


def test_valid_mask_brute_force():
    for spec in fi.tiny_spaces(12, seed0=3000, max_raw=3000):
        assert np.array_equal(oracle.valid_mask(spec), brute.valid_mask(spec)), spec


def test_measured_spaces_node_counts():
    """Node counts of the two single-space workloads, by itertools brute force."""
    spec = fi.single_small()
    assert brute.valid_mask(spec).sum() == oracle.valid_mask(spec).sum() == 832


def test_overflow_and_bad_args():
    big = SpaceSpec("big", ("a", "b"), ((1 << 40, 1), (1 << 40, 2)),
                    (Clause("prod_le", (0, 1), (), 5),))
    with pytest.raises(oracle.OracleError) as e:
        oracle.valid_mask(big)
    assert e.value.code == 2
    bad = SpaceSpec("bad", ("a",), ((1, 2),), (Clause("prod_le", (3,), (), 5),))
    with pytest.raises(oracle.OracleError):
        oracle.valid_mask(bad)


# ---------------------------------------------------------------- neighbourhoods

def test_adjacent_worked_example():
    """Sec. III-B: in [16,32,64,128] the neighbours of 64 are {32,128}, of 128 {64}."""
    rows = _read_golden("adjacent_example.txt")
    values = [int(v) for v in rows[0][1:]]
    spec = _one_param(values)
    for row in rows[1:]:
        centre, expect = int(row[0]), sorted(int(v) for v in row[1:])
        c = values.index(centre)
        f = np.arange(len(values), dtype=np.float64)
        f[c] = 100.0  # the centre is worst, so every neighbour is an out-edge
        g = oracle.build(spec, f, oracle.ADJACENT)
        got = [values[g.node_raw[v]] for v in g.out_idx[g.out_ptr[c]:g.out_ptr[c + 1]]]
        assert got == expect


@pytest.mark.parametrize("nbh", ["hamming", "adjacent"])
def test_ffg_matches_brute_force(nbh):
    code = oracle.HAMMING if nbh == "hamming" else oracle.ADJACENT
    specs = fi.tiny_spaces(10, seed0=5000, max_raw=1500)
    for k, spec in enumerate(specs):
        quantum = 0.5 if k % 3 == 0 else None       # every third space has ties
        f = fi.runtimes(spec, seed=k + 1, fail_frac=0.2 if k % 2 else 0.03, quantum=quantum)
        g = oracle.build(spec, f, code)
        node_raw, outs, ins, failed = brute.edge_lists(spec, f, nbh)
        assert np.array_equal(g.node_raw, node_raw)
        assert np.array_equal(g.failed, failed)
        ptr, idx = brute.csr(outs)
        assert np.array_equal(g.out_ptr, ptr) and np.array_equal(g.out_idx, idx)
        ptr, idx = brute.csr(ins)
        assert np.array_equal(g.in_ptr, ptr) and np.array_equal(g.in_idx, idx)
        is_min = np.array([not failed[v] and len(outs[v]) == 0 for v in range(len(outs))])
        assert np.array_equal(g.is_min, is_min)
        nf = g.node_fit[~g.failed]
        assert g.f_opt == (nf.min() if len(nf) else math.inf)


def test_degree_identities():
    """Distinct fitness, nothing failed: outdeg + indeg = #valid neighbours,
    E = half the degree sum; unconstrained Hamming degree = sum(r_i - 1)."""
    for spec in fi.tiny_spaces(6, seed0=7000, max_raw=2000):
        f = fi.runtimes(spec, seed=3, fail_frac=0.0, noise_sd=0.2)
        assert len(np.unique(f)) == len(f)
        for nbh, code in (("hamming", oracle.HAMMING), ("adjacent", oracle.ADJACENT)):
            g = oracle.build(spec, f, code)
            deg = brute.neighbour_count(spec, nbh)
            indeg = np.diff(g.in_ptr)
            assert np.array_equal(g.outdeg + indeg, deg)
            assert 2 * g.n_edges == deg.sum()
    spec = SpaceSpec("free", ("a", "b", "c"), ((1, 2, 3), (4, 5), (6, 7, 8, 9)))
    g = oracle.build(spec, fi.runtimes(spec, 1, fail_frac=0.0), oracle.HAMMING)
    assert np.all(g.outdeg + np.diff(g.in_ptr) == (3 - 1) + (2 - 1) + (4 - 1))


def test_ties_and_failures():
    """Equal fitness: no edge, both are minima (sink reading).  Failed points
    (fitness 1e10, Sec. V) point to better neighbours, are never minima and
    have no edges among themselves."""
    fail = float(_read_golden("failed_fitness.txt")[0][0])
    spec = _one_param([1, 2, 3, 4])
    g = oracle.build(spec, np.array([2.0, 2.0, fail, fail]), oracle.HAMMING)
    assert g.n_edges == 4                       # 2 -> {0,1}, 3 -> {0,1}
    assert list(g.out_idx) == [0, 1, 0, 1]
    assert list(g.is_min) == [True, True, False, False]
    assert g.f_opt == 2.0
    g = oracle.build(spec, np.array([np.nan, 1.0, 3.0, 1e10]), oracle.ADJACENT)
    assert list(g.failed) == [True, False, False, True]
    assert list(g.is_min) == [False, True, False, False]


def test_global_minimum_is_local_minimum():
    spec = fi.single_small()
    for seed in range(1, 4):
        f = fi.runtimes(spec, seed)
        for code in (oracle.HAMMING, oracle.ADJACENT):
            g = oracle.build(spec, f, code)
            assert g.is_min[np.flatnonzero((g.node_fit == g.f_opt) & ~g.failed)].all()


# ---------------------------------------------------------------- PageRank

def _google_from_graph(g):
    outs = [list(g.out_idx[g.out_ptr[u]:g.out_ptr[u + 1]]) for u in range(g.n_nodes)]
    return outs


@pytest.mark.parametrize("alpha", [0.5, 0.85, 0.95])
def test_pagerank_dense_solve(alpha):
    for k, spec in enumerate(fi.tiny_spaces(5, seed0=9000, max_raw=1500)):
        f = fi.runtimes(spec, seed=k + 11, fail_frac=0.1)
        g = oracle.build(spec, f, oracle.HAMMING if k % 2 else oracle.ADJACENT)
        x_dense = brute.dense_pagerank(_google_from_graph(g), alpha)
        x_exact = oracle.pagerank_exact(g, alpha)
        x_pow, it, res, conv = oracle.pagerank_power(g, alpha, 1e-13)
        assert conv
        assert abs(x_exact.sum() - 1.0) < 1e-13 and abs(x_pow.sum() - 1.0) < 1e-12
        assert np.abs(x_exact - x_dense).sum() < 1e-12
        assert np.abs(x_pow - x_dense).sum() < alpha / (1 - alpha) * res + 1e-13


@pytest.mark.parametrize("alpha", [0.3, 0.85])
def test_chain_closed_form(alpha):
    """1-parameter adjacent space with strictly decreasing fitness: a chain,
    y_k = (1 - alpha^(k+1)) / (1 - alpha), x = y / sum(y)."""
    n = 9
    spec = _one_param(list(range(n)))
    g = oracle.build(spec, np.arange(n, 0, -1, dtype=np.float64), oracle.ADJACENT)
    y = np.array([(1 - alpha ** (k + 1)) / (1 - alpha) for k in range(n)])
    want = y / y.sum()
    assert np.abs(oracle.pagerank_exact(g, alpha) - want).max() < 1e-15
    x, _, _, _ = oracle.pagerank_power(g, alpha, 1e-15)
    assert np.abs(x - want).max() < 1e-14


def test_tournament_closed_form():
    """1-parameter Hamming space, r = 3, distinct fitness: y = (1, 1+a/2, 1+3a/2+a^2/2)."""
    a = 0.85
    spec = _one_param([1, 2, 3])
    g = oracle.build(spec, np.array([3.0, 2.0, 1.0]), oracle.HAMMING)
    y = np.array([1.0, 1 + a / 2, 1 + 1.5 * a + 0.5 * a * a])
    assert np.abs(oracle.pagerank_exact(g, a) - y / y.sum()).max() < 1e-15


@pytest.mark.parametrize("k", [1, 2, 5, 17])
def test_star_closed_forms(k):
    a = 0.85
    # out-star: centre 0 -> leaves 1..k; leaves are dangling
    outs = [list(range(1, k + 1))] + [[] for _ in range(k)]
    ins = [[]] + [[0] for _ in range(k)]
    ptr, idx = brute.csr(ins)
    deg = np.array([len(o) for o in outs])
    key = np.array([2.0] + [1.0] * k)
    want = np.array([1.0] + [1 + a / k] * k) / (1 + k + a)
    assert np.abs(oracle.pagerank_exact_csr(ptr, idx, deg, key, a) - want).max() < 1e-15
    x, _, _ = oracle.pagerank_power_csr(ptr, idx, deg, a, 1e-15)
    assert np.abs(x - want).max() < 1e-14
    # in-star: leaves 1..k -> centre 0
    ins = [list(range(1, k + 1))] + [[] for _ in range(k)]
    ptr, idx = brute.csr(ins)
    deg = np.array([0] + [1] * k)
    key = np.array([1.0] + [2.0] * k)
    want = np.array([1 + a * k] + [1.0] * k) / (1 + k + a * k)
    assert np.abs(oracle.pagerank_exact_csr(ptr, idx, deg, key, a) - want).max() < 1e-15
    x, _, _ = oracle.pagerank_power_csr(ptr, idx, deg, a, 1e-15)
    assert np.abs(x - want).max() < 1e-14


def test_pagerank_networkx():
    """Cross-check against networkx.pagerank (uniform teleport and dangling)."""
    nx = pytest.importorskip("networkx")
    spec = fi.single_small()
    f = fi.runtimes(spec, 4)
    g = oracle.build(spec, f, oracle.HAMMING)
    G = nx.DiGraph()
    G.add_nodes_from(range(g.n_nodes))
    for u in range(g.n_nodes):
        for v in g.out_idx[g.out_ptr[u]:g.out_ptr[u + 1]]:
            G.add_edge(u, int(v))
    pr = nx.pagerank(G, alpha=0.85, tol=1e-15, max_iter=10000)
    ref = np.array([pr[v] for v in range(g.n_nodes)])
    assert np.abs(oracle.pagerank_exact(g, 0.85) - ref).sum() < 1e-10


def test_power_contraction_bound_large():
    """||x_k - x*||_1 <= alpha/(1-alpha) * residual_k on a full-size space."""
    spec = fi.single_small()
    f = fi.runtimes(spec, 7, fail_frac=0.3)
    g = oracle.build(spec, f, oracle.HAMMING)
    xe = oracle.pagerank_exact(g, 0.85)
    for tol in (1e-4, 1e-8, 1e-12):
        x, it, res, conv = oracle.pagerank_power(g, 0.85, tol)
        assert conv and res < tol
        assert np.abs(x - xe).sum() <= 0.85 / 0.15 * res + 1e-14


def test_alpha_to_zero_uniform():
    spec = fi.single_small()
    g = oracle.build(spec, fi.runtimes(spec, 2), oracle.HAMMING)
    x = oracle.pagerank_exact(g, 0.0)
    assert np.abs(x - 1.0 / g.n_nodes).max() < 1e-18


# ---------------------------------------------------------------- C_p

def test_centrality_hand_example():
    """Three minima with fitness 1.0, 1.04, 1.5 and ranks 0.2, 0.3, 0.5:
    C_0 = 0.2, C_0.05 = 0.5, C_0.5 = 1 (threshold f <= (1+p) f_opt)."""
    class G:
        pass
    g = G()
    g.n_nodes = 5
    g.is_min = np.array([True, False, True, True, False])
    g.node_fit = np.array([1.0, 0.5, 1.04, 1.5, 9.0])   # node 1 is not a minimum
    g.f_opt = 1.0
    x = np.array([0.2, 0.7, 0.3, 0.5, 0.1])
    cp = oracle.centrality(g, x, [0.0, 0.03, 0.05, 0.49, 0.5, 10.0])
    assert np.allclose(cp, [0.2, 0.2, 0.5, 0.5, 1.0, 1.0], rtol=0, atol=1e-16)


def test_centrality_properties():
    spec = fi.single_large()
    small = fi.single_small()
    f = fi.runtimes(small, 5, fail_frac=0.2)
    g = oracle.build(small, f, oracle.HAMMING)
    x = oracle.pagerank_exact(g, 0.85)
    ps = np.linspace(0, 1.0, 41)
    cp = oracle.centrality(g, x, ps)
    assert np.all(np.diff(cp) >= 0)                       # monotone in p
    pmax = g.node_fit[g.is_min].max() / g.f_opt - 1
    assert oracle.centrality(g, x, [pmax * 1.0001])[0] == 1.0
    assert np.allclose(oracle.centrality(g, 7.5 * x, ps), cp, rtol=1e-15, atol=1e-15)
    # alpha -> 0: ranks are uniform, C_p = |L_p| / |L|
    x0 = oracle.pagerank_exact(g, 0.0)
    minf = g.node_fit[g.is_min]
    frac = [(minf <= g.f_opt * (1 + p)).sum() / len(minf) for p in ps]
    assert np.allclose(oracle.centrality(g, x0, ps), frac, rtol=0, atol=1e-15)
    # a single minimum: C_p = 1 for every p
    chain = _one_param(list(range(6)))
    gc = oracle.build(chain, np.arange(6, 0, -1, dtype=np.float64), oracle.ADJACENT)
    assert np.all(oracle.centrality(gc, oracle.pagerank_exact(gc), ps) == 1.0)
    assert spec.n_raw == 2162688


# ---------------------------------------------------------------- exact DAG solve, absorbing walk

def _dense_A(g):
    """A[v, u] = 1/outdeg(u) for every edge u -> v."""
    A = np.zeros((g.n_nodes, g.n_nodes))
    for u in range(g.n_nodes):
        for v in g.out_idx[g.out_ptr[u]:g.out_ptr[u + 1]]:
            A[v, u] += 1.0 / g.outdeg[u]
    return A


@pytest.mark.parametrize("d", [0.0, 0.5, 0.85, 1.0])
def test_dag_values_dense_solve(d):
    """(I - d A) y = 1 solved densely; y / sum y is the exact PageRank."""
    for k, spec in enumerate(fi.tiny_spaces(5, seed0=9100, max_raw=1200)):
        f = fi.runtimes(spec, seed=k + 31, fail_frac=(0.03, 0.3, 0.7)[k % 3])
        g = oracle.build(spec, f, oracle.HAMMING if k % 2 else oracle.ADJACENT)
        y = oracle.dag_values(g, d)
        ref = np.linalg.solve(np.eye(g.n_nodes) - d * _dense_A(g), np.ones(g.n_nodes))
        assert np.abs(y - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
        if d < 1.0:
            assert np.abs(y / y.sum() - oracle.pagerank_exact(g, d)).sum() < 1e-14


def test_absorption_dense_solve_and_mass():
    """(I - A) a = 1/n; every walk ends at a node without out-edges, so their
    probabilities sum to 1."""
    for k, spec in enumerate(fi.tiny_spaces(6, seed0=9200, max_raw=1500)):
        f = fi.runtimes(spec, seed=k + 41, fail_frac=(0.03, 0.3, 0.7)[k % 3],
                        quantum=0.5 if k % 2 else None)
        g = oracle.build(spec, f, oracle.HAMMING if k % 2 else oracle.ADJACENT)
        a = oracle.absorption(g)
        n = g.n_nodes
        ref = np.linalg.solve(np.eye(n) - _dense_A(g), np.full(n, 1.0 / n))
        assert np.abs(a - ref).max() < 1e-13
        assert abs(a[g.outdeg == 0].sum() - 1.0) < 1e-13
        assert (a >= 1.0 / n - 1e-15).all()     # every node is at least a start


def test_absorption_closed_forms():
    # chain 0 -> 1 -> ... -> n-1 (strictly decreasing fitness): a_k = (k+1)/n,
    # the last node collects every walk
    n = 7
    spec = _one_param(list(range(n)))
    g = oracle.build(spec, np.arange(n, 0, -1, dtype=np.float64), oracle.ADJACENT)
    assert np.abs(oracle.absorption(g) - np.arange(1, n + 1) / n).max() < 1e-15
    # out-star: centre -> k leaves, each leaf 1/n + (1/n)/k
    for k in (1, 3, 8):
        ins = [[]] + [[0] for _ in range(k)]
        ptr, idx = brute.csr(ins)
        deg = np.array([k] + [0] * k)
        key = np.array([2.0] + [1.0] * k)
        n = k + 1
        want = np.array([1.0 / n] + [1.0 / n + 1.0 / (n * k)] * k)
        assert np.abs(oracle.absorption_csr(ptr, idx, deg, key) - want).max() < 1e-15
    # in-star: k leaves -> centre: the centre collects everything
    k = 5
    ins = [list(range(1, k + 1))] + [[] for _ in range(k)]
    ptr, idx = brute.csr(ins)
    deg = np.array([0] + [1] * k)
    key = np.array([1.0] + [2.0] * k)
    a = oracle.absorption_csr(ptr, idx, deg, key)
    assert abs(a[0] - 1.0) < 1e-15 and np.abs(a[1:] - 1.0 / (k + 1)).max() < 1e-15


# ---------------------------------------------------------------- simulated improving walks

def test_splitmix64_reference_outputs():
    """The first outputs of SplitMix64 from state 0 (the published reference
    sequence)."""
    g = 0x9E3779B97F4A7C15
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [oracle.splitmix64((k * g) & 0xFFFFFFFFFFFFFFFF) for k in range(3)] == want


def test_walks_chain_and_mass():
    n = 6
    spec = _one_param(list(range(n)))
    g = oracle.build(spec, np.arange(n, 0, -1, dtype=np.float64), oracle.ADJACENT)
    counts, steps = oracle.walks(g, seed=3, n_walks=1000)
    assert counts[-1] == 1000 and counts[:-1].sum() == 0
    # a walk from node k makes n-1-k moves; starts are uniform
    assert 0 < steps < 1000 * (n - 1)


def test_walk_frequencies_match_absorption():
    """Arrival frequencies of 200,000 walks against the exact arrival
    probabilities, within 5 binomial standard deviations at every sink."""
    spaces = [fi.single_small(), fi.conv_mi50_space()] + fi.tiny_spaces(3, seed0=9300,
                                                                         max_raw=1500)
    for k, spec in enumerate(spaces):
        f = fi.runtimes(spec, seed=k + 51, fail_frac=(0.03, 0.3)[k % 2])
        g = oracle.build(spec, f, oracle.HAMMING if k % 2 else oracle.ADJACENT)
        W = 200_000
        counts, _ = oracle.walks(g, seed=100 + k, n_walks=W)
        a = oracle.absorption(g)
        sinks = g.outdeg == 0
        assert counts[~sinks].sum() == 0 and counts.sum() == W
        p = a[sinks]
        freq = counts[sinks] / W
        sd = np.sqrt(np.clip(p * (1 - p), 0.0, None) / W)
        assert (np.abs(freq - p) <= 5 * sd + 1e-12).all()


def test_minima_fraction():
    """Hand example: fitness 4 (min), 6, 2 (min, optimum), 5 on an adjacent
    line: minima 0 and 2 give 2/4 and 2/2."""
    spec = _one_param([1, 2, 3, 4])
    g = oracle.build(spec, np.array([4.0, 6.0, 2.0, 5.0]), oracle.ADJACENT)
    assert list(g.is_min) == [True, False, True, False]
    assert list(oracle.minima_fraction(g)) == [0.5, 1.0]
    for seed in (1, 2):
        g = oracle.build(fi.single_small(), fi.runtimes(fi.single_small(), seed), oracle.HAMMING)
        fr = oracle.minima_fraction(g)
        assert len(fr) == g.is_min.sum() and (fr > 0).all() and (fr <= 1).all()
        assert (fr == 1.0).any()
