"""CPU oracle of the fitness-flow-graph metric (ctypes front end of ffg_oracle.c).

TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the
benchmark's CPU-baseline leg may import this package; the library
``paper_2210_01465_gb300`` never does, and this package never imports the
library.  The two share no source: the C oracle has its own header, its own
space layout and its own constants.

What each function computes (all FP64, single-threaded, plain loops):

* ``valid_mask``   -- which points of X = S_1 x ... x S_n satisfy every
                      clause (Sec. III-B).
* ``build``        -- the FFG (Sec. VII-B): nodes = valid points ranked by raw
                      index; edge u->v iff v is a neighbour of u (Hamming,
                      Eq. 2, or adjacent-value, Sec. III-B) with strictly lower
                      fitness; failed points (fitness not below 1e10, Sec. V)
                      compare as +inf and are never minima; both out- and
                      in-lists sorted by node id.
* ``pagerank_power`` -- damped power iteration on the column-normalised
                      adjacency matrix (Sec. VII-B) with uniform teleport and
                      uniform dangling redistribution, L1 stopping rule.
* ``pagerank_exact`` -- the same fixed point solved directly on the DAG.
* ``centrality``   -- C_p of Sec. VII-B (Eq. 3), compensated FP64 sums.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ffg_oracle.c")
_HDR = os.path.join(_HERE, "ffg_oracle.h")
LIB_PATH = os.path.join(_HERE, "libffg_oracle.so")
_TEST_SRC = os.path.join(_HERE, "test_oracle.c")
TEST_EXE = os.path.join(_HERE, "test_oracle")

HAMMING, ADJACENT = 0, 1
_KIND = {"prod_le": 0, "prod_ge": 1, "divides": 2, "prod_le_prod": 3}
_STATUS = {0: "ok", 1: "bad argument", 2: "overflow", 3: "out of memory", 4: "not converged",
           5: "empty"}


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"oracle {what}: {_STATUS.get(code, code)}")
        self.code = code


def compile_oracle(force: bool = False) -> str:
    """Compile ffg_oracle.c with gcc into a shared library next to it, and the
    C self-test (``test_oracle.c``) into an executable beside it."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < newest:
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fno-fast-math",
                        "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, LIB_PATH)
    compile_self_test(force)
    return LIB_PATH


def compile_self_test(force: bool = False) -> str:
    """Compile the oracle's C self-test (test_oracle.c + ffg_oracle.c)."""
    newest = max(os.path.getmtime(p) for p in (_SRC, _HDR, _TEST_SRC))
    if not force and os.path.exists(TEST_EXE) and os.path.getmtime(TEST_EXE) >= newest:
        return TEST_EXE
    tmp = TEST_EXE + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fno-fast-math",
                    "-I", _HERE, "-o", tmp, _TEST_SRC, _SRC, "-lm"], check=True)
    os.replace(tmp, TEST_EXE)
    return TEST_EXE


def run_self_test() -> tuple[int, str]:
    """Run the C self-test; returns (exit status, its output)."""
    exe = compile_self_test()
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    return r.returncode, r.stdout + r.stderr


class _Clause(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_a", C.c_int32), ("n_b", C.c_int32),
                ("a", C.c_int32 * 16), ("b", C.c_int32 * 16), ("bound", C.c_int64)]


class _Space(C.Structure):
    _fields_ = [("n_params", C.c_int32), ("radix", C.POINTER(C.c_int32)),
                ("values", C.POINTER(C.c_int64)), ("n_clauses", C.c_int32),
                ("clauses", C.POINTER(_Clause))]


class _Graph(C.Structure):
    _fields_ = [("n_raw", C.c_int64), ("n_nodes", C.c_int64), ("n_edges", C.c_int64),
                ("node_raw", C.POINTER(C.c_int64)), ("out_ptr", C.POINTER(C.c_int64)),
                ("out_idx", C.POINTER(C.c_int32)), ("in_ptr", C.POINTER(C.c_int64)),
                ("in_idx", C.POINTER(C.c_int32)), ("outdeg", C.POINTER(C.c_int32)),
                ("is_min", C.POINTER(C.c_uint8)), ("failed", C.POINTER(C.c_uint8)),
                ("node_fit", C.POINTER(C.c_double)), ("f_opt", C.c_double)]


_lib = None
_lock = threading.Lock()


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(compile_oracle())
            P = C.POINTER
            lib.or_raw_count.argtypes = [P(_Space), P(C.c_int64)]
            lib.or_valid_mask.argtypes = [P(_Space), C.c_void_p]
            lib.or_build.argtypes = [P(_Space), C.c_void_p, C.c_int, C.c_double, P(_Graph)]
            lib.or_graph_free.argtypes = [P(_Graph)]
            lib.or_graph_free.restype = None
            lib.or_pagerank_power.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.c_double, C.c_double, C.c_int32, C.c_void_p,
                                              P(C.c_int32), P(C.c_double)]
            lib.or_pagerank_exact.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]
            lib.or_centrality.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_double, C.c_void_p, C.c_int32, C.c_void_p]
            lib.or_dag_values.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]
            lib.or_absorption.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_void_p]
            lib.or_minima_fraction.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_double,
                                               C.c_void_p, C.POINTER(C.c_int64)]
            lib.or_splitmix64.restype = C.c_uint64
            lib.or_splitmix64.argtypes = [C.c_uint64]
            lib.or_walks.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64,
                                     C.c_int64, C.c_void_p, C.POINTER(C.c_int64)]
            _lib = lib
    return _lib


class _SpaceHolder:
    """Keeps the ctypes arrays of one space alive while the C code reads them."""

    def __init__(self, spec):
        self.radix = np.ascontiguousarray([len(v) for v in spec.values], dtype=np.int32)
        flat = [int(x) for v in spec.values for x in v]
        self.values = np.ascontiguousarray(flat if flat else [0], dtype=np.int64)
        n_cl = len(spec.clauses)
        self.clauses = (_Clause * max(n_cl, 1))()
        for k, cl in enumerate(spec.clauses):
            c = self.clauses[k]
            c.kind = _KIND[cl.kind]
            c.n_a, c.n_b = len(cl.a), len(cl.b)
            for t, i in enumerate(sorted(cl.a)):
                c.a[t] = i
            for t, i in enumerate(sorted(cl.b)):
                c.b[t] = i
            c.bound = int(cl.bound)
        self.s = _Space(len(spec.values), self.radix.ctypes.data_as(C.POINTER(C.c_int32)),
                        self.values.ctypes.data_as(C.POINTER(C.c_int64)), n_cl,
                        C.cast(self.clauses, C.POINTER(_Clause)))


def _ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data)


def raw_count(spec) -> int:
    h = _SpaceHolder(spec)
    r = C.c_int64()
    st = _load().or_raw_count(C.byref(h.s), C.byref(r))
    if st:
        raise OracleError(st, "raw_count")
    return int(r.value)


def valid_mask(spec) -> np.ndarray:
    h = _SpaceHolder(spec)
    out = np.zeros(raw_count(spec), dtype=np.uint8)
    st = _load().or_valid_mask(C.byref(h.s), _ptr(out))
    if st:
        raise OracleError(st, "valid_mask")
    return out.astype(bool)


class Graph:
    """FFG arrays as numpy copies (see ``build``)."""

    def __init__(self, g: _Graph):
        N, E = int(g.n_nodes), int(g.n_edges)
        cp = lambda p, n, dt: np.ctypeslib.as_array(p, shape=(n,)).astype(dt, copy=True) \
            if n > 0 else np.zeros(0, dtype=dt)  # noqa: E731
        self.n_raw, self.n_nodes, self.n_edges = int(g.n_raw), N, E
        self.node_raw = cp(g.node_raw, N, np.int64)
        self.out_ptr = cp(g.out_ptr, N + 1, np.int64)
        self.in_ptr = cp(g.in_ptr, N + 1, np.int64)
        self.out_idx = cp(g.out_idx, E, np.int32)
        self.in_idx = cp(g.in_idx, E, np.int32)
        self.outdeg = cp(g.outdeg, N, np.int32)
        self.is_min = cp(g.is_min, N, np.uint8).astype(bool)
        self.failed = cp(g.failed, N, np.uint8).astype(bool)
        self.node_fit = cp(g.node_fit, N, np.float64)
        self.f_opt = float(g.f_opt)


def build(spec, fitness_raw: np.ndarray, nbh: int = HAMMING, fail_thr: float = 1e10) -> Graph:
    h = _SpaceHolder(spec)
    f = np.ascontiguousarray(fitness_raw, dtype=np.float64)
    if f.shape != (spec.n_raw,):
        raise ValueError("fitness_raw must hold one value per raw point")
    g = _Graph()
    lib = _load()
    st = lib.or_build(C.byref(h.s), _ptr(f), int(nbh), float(fail_thr), C.byref(g))
    try:
        if st:
            raise OracleError(st, "build")
        return Graph(g)
    finally:
        lib.or_graph_free(C.byref(g))


def pagerank_power(g: Graph, alpha: float = 0.85, tol: float = 1e-12, max_iter: int = 10000):
    """Returns (x, iters, residual, converged)."""
    x = np.zeros(max(g.n_nodes, 1), dtype=np.float64)
    it, res = C.c_int32(), C.c_double()
    st = _load().or_pagerank_power(g.n_nodes, _ptr(g.in_ptr), _ptr(g.in_idx), _ptr(g.outdeg),
                                   alpha, tol, max_iter, _ptr(x), C.byref(it), C.byref(res))
    if st not in (0, 4):
        raise OracleError(st, "pagerank_power")
    return x[:g.n_nodes], int(it.value), float(res.value), st == 0


def pagerank_exact(g: Graph, alpha: float = 0.85) -> np.ndarray:
    x = np.zeros(max(g.n_nodes, 1), dtype=np.float64)
    failed = g.failed.astype(np.uint8)
    st = _load().or_pagerank_exact(g.n_nodes, _ptr(g.in_ptr), _ptr(g.in_idx), _ptr(g.outdeg),
                                   _ptr(failed), _ptr(g.node_fit), alpha, _ptr(x))
    if st:
        raise OracleError(st, "pagerank_exact")
    return x[:g.n_nodes]


def dag_values(g: Graph, d: float) -> np.ndarray:
    """y[v] = 1 + d * sum_{u -> v} y[u] / outdeg[u] (unnormalised exact solve)."""
    y = np.zeros(max(g.n_nodes, 1), dtype=np.float64)
    failed = g.failed.astype(np.uint8)
    st = _load().or_dag_values(g.n_nodes, _ptr(g.in_ptr), _ptr(g.in_idx), _ptr(g.outdeg),
                               _ptr(failed), _ptr(g.node_fit), d, _ptr(y))
    if st:
        raise OracleError(st, "dag_values")
    return y[:g.n_nodes]


def absorption(g: Graph) -> np.ndarray:
    """Probability that an improving walk from a uniform start passes / ends
    at each node."""
    a = np.zeros(max(g.n_nodes, 1), dtype=np.float64)
    failed = g.failed.astype(np.uint8)
    st = _load().or_absorption(g.n_nodes, _ptr(g.in_ptr), _ptr(g.in_idx), _ptr(g.outdeg),
                               _ptr(failed), _ptr(g.node_fit), _ptr(a))
    if st:
        raise OracleError(st, "absorption")
    return a[:g.n_nodes]


def dag_values_csr(in_ptr, in_idx, outdeg, key, d):
    """``key``: per-node fitness; edges must run from higher to lower key."""
    in_ptr = np.ascontiguousarray(in_ptr, dtype=np.int64)
    in_idx = np.ascontiguousarray(in_idx if len(in_idx) else [0], dtype=np.int32)
    outdeg = np.ascontiguousarray(outdeg, dtype=np.int32)
    key = np.ascontiguousarray(key, dtype=np.float64)
    n = len(outdeg)
    failed = np.zeros(n, dtype=np.uint8)
    y = np.zeros(n, dtype=np.float64)
    st = _load().or_dag_values(n, _ptr(in_ptr), _ptr(in_idx), _ptr(outdeg), _ptr(failed),
                               _ptr(key), d, _ptr(y))
    if st:
        raise OracleError(st, "dag_values")
    return y


def absorption_csr(in_ptr, in_idx, outdeg, key):
    in_ptr = np.ascontiguousarray(in_ptr, dtype=np.int64)
    in_idx = np.ascontiguousarray(in_idx if len(in_idx) else [0], dtype=np.int32)
    outdeg = np.ascontiguousarray(outdeg, dtype=np.int32)
    key = np.ascontiguousarray(key, dtype=np.float64)
    n = len(outdeg)
    failed = np.zeros(n, dtype=np.uint8)
    a = np.zeros(n, dtype=np.float64)
    st = _load().or_absorption(n, _ptr(in_ptr), _ptr(in_idx), _ptr(outdeg), _ptr(failed),
                               _ptr(key), _ptr(a))
    if st:
        raise OracleError(st, "absorption")
    return a


def minima_fraction(g: Graph) -> np.ndarray:
    """f_opt / f(x) of every local minimum (ascending node order)."""
    out = np.zeros(max(g.n_nodes, 1), dtype=np.float64)
    k = C.c_int64(0)
    is_min = g.is_min.astype(np.uint8)
    st = _load().or_minima_fraction(g.n_nodes, _ptr(is_min), _ptr(g.node_fit), g.f_opt,
                                    _ptr(out), C.byref(k))
    if st:
        raise OracleError(st, "minima_fraction")
    return out[:k.value]


def splitmix64(x: int) -> int:
    return int(_load().or_splitmix64(int(x) & 0xFFFFFFFFFFFFFFFF))


def walks_csr(out_ptr, out_idx, outdeg, seed: int, n_walks: int):
    """Simulated improving walks; returns (counts per node, total steps)."""
    out_ptr = np.ascontiguousarray(out_ptr, dtype=np.int64)
    out_idx = np.ascontiguousarray(out_idx if len(out_idx) else [0], dtype=np.int32)
    outdeg = np.ascontiguousarray(outdeg, dtype=np.int32)
    n = len(outdeg)
    counts = np.zeros(n, dtype=np.uint64)
    steps = C.c_int64(0)
    st = _load().or_walks(n, _ptr(out_ptr), _ptr(out_idx), _ptr(outdeg),
                          int(seed) & 0xFFFFFFFFFFFFFFFF, int(n_walks), _ptr(counts),
                          C.byref(steps))
    if st:
        raise OracleError(st, "walks")
    return counts, int(steps.value)


def walks(g: Graph, seed: int, n_walks: int):
    return walks_csr(g.out_ptr, g.out_idx, g.outdeg, seed, n_walks)


def centrality(g: Graph, x: np.ndarray, p) -> np.ndarray:
    pv = np.ascontiguousarray(p, dtype=np.float64)
    xs = np.ascontiguousarray(x, dtype=np.float64)
    is_min = g.is_min.astype(np.uint8)
    out = np.zeros(max(len(pv), 1), dtype=np.float64)
    st = _load().or_centrality(g.n_nodes, _ptr(is_min), _ptr(g.node_fit), _ptr(xs), g.f_opt,
                               _ptr(pv), len(pv), _ptr(out))
    if st:
        raise OracleError(st, "centrality")
    return out[:len(pv)]


# generic PageRank pieces the tests use for pins on hand-made graphs
def pagerank_power_csr(in_ptr, in_idx, outdeg, alpha=0.85, tol=1e-14, max_iter=100000):
    in_ptr = np.ascontiguousarray(in_ptr, dtype=np.int64)
    in_idx = np.ascontiguousarray(in_idx if len(in_idx) else [0], dtype=np.int32)
    outdeg = np.ascontiguousarray(outdeg, dtype=np.int32)
    n = len(outdeg)
    x = np.zeros(n, dtype=np.float64)
    it, res = C.c_int32(), C.c_double()
    st = _load().or_pagerank_power(n, _ptr(in_ptr), _ptr(in_idx), _ptr(outdeg), alpha, tol,
                                   max_iter, _ptr(x), C.byref(it), C.byref(res))
    if st not in (0, 4):
        raise OracleError(st, "pagerank_power")
    return x, int(it.value), float(res.value)


def pagerank_exact_csr(in_ptr, in_idx, outdeg, key, alpha=0.85):
    """``key``: per-node fitness; edges must run from higher to lower key."""
    in_ptr = np.ascontiguousarray(in_ptr, dtype=np.int64)
    in_idx = np.ascontiguousarray(in_idx if len(in_idx) else [0], dtype=np.int32)
    outdeg = np.ascontiguousarray(outdeg, dtype=np.int32)
    key = np.ascontiguousarray(key, dtype=np.float64)
    n = len(outdeg)
    failed = np.zeros(n, dtype=np.uint8)
    x = np.zeros(n, dtype=np.float64)
    st = _load().or_pagerank_exact(n, _ptr(in_ptr), _ptr(in_idx), _ptr(outdeg), _ptr(failed),
                                   _ptr(key), alpha, _ptr(x))
    if st:
        raise OracleError(st, "pagerank_exact")
    return x
