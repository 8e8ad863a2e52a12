"""Fitness flow graphs, PageRank and proportion of centrality on GB300.

Python binding of the C ABI in ``include/ffg.h`` (library
``lib/libffg_gb300.so``, CUDA kernels for sm_103a).  This module only
marshals arguments: every step of the computation -- the FFG build of
Sec. VII-B over the neighbourhoods of Sec. III-B, PageRank, and C_p of
Sec. VII-B (Eq. 3) -- runs in the library's kernels.  PyTorch provides
device memory and streams.  There is no CPU fallback: if the library is
missing, loading it raises.

Two layers:

* same-name wrappers of the C functions (``ffg_build_count``,
  ``ffg_build_fill``, ``pagerank_solve``, ``pagerank_query``,
  ``centrality_proportion``, the ``*_workspace_bytes`` queries and the
  diagnostics), taking device pointers as integers;
* tensor helpers (``Space``, ``build_graph``, ``pagerank``, ``centrality``)
  that allocate workspaces and outputs with torch and call the wrappers.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from ._build import CHECKED_LIB_PATH, LIB_PATH, build  # noqa: F401

# ---- constants of include/ffg.h -------------------------------------------
FFG_OK, FFG_ERR_INVALID_ARG, FFG_ERR_OVERFLOW, FFG_ERR_CUDA = 0, 1, 2, 3
FFG_ERR_EMPTY, FFG_ERR_NOT_CONVERGED, FFG_ERR_TIMEOUT, FFG_ERR_NO_MEMORY = 4, 5, 6, 7
HAMMING, ADJACENT = 0, 1
F64, F32 = 0, 1
PROD_LE, PROD_GE, DIVIDES, PROD_LE_PROD = 0, 1, 2, 3
INIT_RANKS, INIT_LAYOUT = 1, 2
MAX_ITER = 1000000  # FFG_MAX_ITER
MAX_PARAMS, MAX_VALUES, MAX_CONSTRAINTS, MAX_P = 16, 1024, 16, 32
_KIND = {"prod_le": PROD_LE, "prod_ge": PROD_GE, "divides": DIVIDES,
         "prod_le_prod": PROD_LE_PROD}


class FFGError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        detail = ffg_last_error()
        super().__init__(f"{where}: {ffg_status_str(status)}" + (f" ({detail})" if detail else ""))


class ffg_constraint(C.Structure):
    _fields_ = [("kind", C.c_int32), ("mask_a", C.c_uint32), ("mask_b", C.c_uint32),
                ("reserved", C.c_int32), ("bound", C.c_int64)]


class ffg_space(C.Structure):
    _fields_ = [("n_params", C.c_int32), ("radix", C.POINTER(C.c_int32)),
                ("values", C.POINTER(C.c_int64)), ("n_constraints", C.c_int32),
                ("constraints", C.POINTER(ffg_constraint))]


class ffg_graph(C.Structure):
    _fields_ = [("n_raw", C.c_int64), ("n_nodes", C.c_int64), ("n_edges", C.c_int64),
                ("n_minima", C.c_int64), ("out_ptr", C.c_void_p), ("out_idx", C.c_void_p),
                ("in_ptr", C.c_void_p), ("in_idx", C.c_void_p), ("outdeg", C.c_void_p),
                ("node_raw", C.c_void_p), ("is_min", C.c_void_p), ("f_opt", C.c_double)]


class ffg_pr_job(C.Structure):
    _fields_ = [("g", C.POINTER(ffg_graph)), ("damping", C.c_double), ("tol", C.c_double),
                ("max_iter", C.c_int32), ("init", C.c_int32), ("ranks", C.c_void_p)]


PARAM_JOBS = 240  # FFG_PR_PARAM_JOBS: batches up to this size pass their job table as parameters


class ffg_pr_batch(C.Structure):
    _fields_ = [("prec", C.c_int32), ("n_jobs", C.c_int32), ("n_graphs", C.c_int32),
                ("n_blocks", C.c_int32), ("warps", C.c_int32), ("n_items", C.c_int32),
                ("claim", C.c_int32), ("w_form", C.c_int32),
                ("total_tiles", C.c_int64), ("jobs", C.c_void_p),
                ("graphs", C.c_void_p), ("items", C.c_void_p), ("first", C.c_void_p),
                ("queue", C.c_void_p),
                ("ctl", C.c_void_p), ("total_rows", C.c_int64), ("tables", C.c_void_p * 10),
                ("param_jobs", C.c_int32), ("reserved", C.c_int32),
                ("params", C.c_uint64 * (PARAM_JOBS * 16))]


class ffg_build_job(C.Structure):
    _fields_ = [("space", C.POINTER(ffg_space)), ("fitness_raw", C.c_void_p),
                ("nbh", C.c_int32), ("reserved", C.c_int32), ("fail_thr", C.c_double),
                ("g", C.POINTER(ffg_graph))]


class ffg_build_batch(C.Structure):
    _fields_ = [("n_jobs", C.c_int32), ("reserved", C.c_int32), ("total_raw", C.c_int64),
                ("total_words", C.c_int64), ("total_blocks", C.c_int64),
                ("total_rows", C.c_int64), ("tables", C.c_void_p * 20)]


class ffg_pr_tuning(C.Structure):
    _fields_ = [("split", C.c_double), ("grain", C.c_double), ("max_blocks", C.c_int32),
                ("block_warps", C.c_int32), ("claim", C.c_int32), ("fp64_form", C.c_int32),
                ("min_tiles", C.c_int32), ("reserved", C.c_int32),
                ("job_cost", C.POINTER(C.c_double))]


class ffg_cp_job(C.Structure):
    _fields_ = [("g", C.POINTER(ffg_graph)), ("fitness_raw", C.c_void_p), ("ranks", C.c_void_p)]


class ffg_rows_op(C.Structure):
    _fields_ = [("op", C.c_int32), ("max_iter", C.c_int32), ("damping", C.c_double),
                ("tol", C.c_double), ("w_in", C.c_void_p), ("w_out", C.c_void_p),
                ("ranks", C.c_void_p), ("sums", C.c_void_p), ("ctl", C.c_void_p)]


ROWS_INIT, ROWS_STEP, ROWS_SUM, ROWS_WRITE = 0, 1, 2, 3
ROWS_START, ROWS_ADVANCE, ROWS_SCALE = 4, 5, 6
ROWS_CTL_BYTES = 48   # sizeof(ffg_rows_ctl): iters, stop, converged, status (int32),
                      # residual, prev_residual, scale (double), dangling (uint64)


class ffg_cp_batch(C.Structure):
    _fields_ = [("n_jobs", C.c_int32), ("n_p", C.c_int32), ("prec", C.c_int32),
                ("reserved", C.c_int32), ("cp", C.c_void_p), ("status", C.c_void_p),
                ("tables", C.c_void_p * 8)]


class ffg_batch_desc(C.Structure):
    _fields_ = [("build", C.POINTER(ffg_build_batch)), ("pagerank", C.POINTER(ffg_pr_batch)),
                ("cp", C.POINTER(ffg_cp_batch))]


class ffg_batch_out(C.Structure):
    _fields_ = [("build_status", C.c_void_p), ("iters", C.c_void_p), ("residual", C.c_void_p),
                ("pr_status", C.c_void_p), ("cp", C.c_void_p)]


# names of include/ffg.h's entry points (the ABI test checks the header)
ENTRY_POINTS = ("ffg_workspace_bytes", "ffg_build_count", "ffg_build_fill",
                "ffg_build_batch_workspace_bytes", "ffg_build_batch_count",
                "ffg_build_batch_fill", "ffg_build_batch_rerun", "ffg_build_batch_query",
                "pagerank_workspace_bytes", "pagerank_prepare", "pagerank_solve",
                "pagerank_solve_static",
                "pagerank_query", "dag_workspace_bytes", "dag_solve",
                "walk_workspace_bytes", "walk_simulate",
                "minima_workspace_bytes", "minima_fraction",
                "pagerank_batch_workspace_bytes", "pagerank_batch_plan",
                "pagerank_batch_plan_tuned",
                "pagerank_batch_run", "pagerank_batch_prepare", "pagerank_batch_solve",
                "pagerank_batch_query", "pagerank_batch_times",
                "pagerank_rows_w_bytes", "pagerank_rows_workspace_bytes",
                "pagerank_rows_prepare", "pagerank_rows_run",
                "centrality_workspace_bytes", "centrality_proportion",
                "centrality_batch_workspace_bytes", "centrality_batch_plan",
                "centrality_batch_run", "centrality_batch_query", "centrality_batch",
                "ffg_batch_run",
                "ffg_status_str",
                "ffg_last_error", "ffg_launch_count",
                "ffg_checked_build", "ffg_checked_failures")

_lib = None


def default_lib_path() -> str:
    """The library ``load()`` opens: ``FFG_LIB=checked`` selects the
    bounds-checked build, another non-empty value is a path."""
    sel = os.environ.get("FFG_LIB", "")
    if sel == "checked":
        return CHECKED_LIB_PATH
    return sel or LIB_PATH


def load(path: str | None = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or default_lib_path()
    if not os.path.exists(p):
        raise ImportError(f"FFG CUDA library not built: {p} is missing "
                          "(run paper_2210_01465_gb300.build())")
    lib = C.CDLL(p)
    P = C.POINTER
    vp, i32, i64, f64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_size_t
    lib.ffg_workspace_bytes.argtypes = [P(ffg_space), C.c_int]
    lib.ffg_workspace_bytes.restype = sz
    lib.ffg_build_count.argtypes = [P(ffg_space), vp, C.c_int, f64, P(ffg_graph), P(i64), P(i64),
                                    vp, sz, vp]
    lib.ffg_build_fill.argtypes = [P(ffg_space), vp, C.c_int, f64, P(ffg_graph), vp, sz, vp]
    lib.pagerank_workspace_bytes.argtypes = [i64, i64, C.c_int]
    lib.pagerank_workspace_bytes.restype = sz
    lib.pagerank_solve.argtypes = [P(ffg_graph), f64, f64, i32, C.c_int, vp, C.c_int, vp, sz,
                                   P(i32), P(f64), vp]
    lib.pagerank_prepare.argtypes = [P(ffg_graph), C.c_int, vp, sz, vp]
    lib.pagerank_solve_static.argtypes = [P(ffg_graph), f64, f64, i32, C.c_int, vp, C.c_int,
                                          P(i32), P(f64), vp]
    lib.pagerank_query.argtypes = [vp, P(i32), P(f64), vp]
    lib.pagerank_batch_workspace_bytes.argtypes = [P(ffg_pr_job), i32, C.c_int]
    lib.pagerank_batch_workspace_bytes.restype = sz
    lib.pagerank_batch_plan.argtypes = [P(ffg_pr_job), i32, C.c_int, vp, sz, P(ffg_pr_batch), vp]
    lib.minima_workspace_bytes.restype = sz
    lib.minima_workspace_bytes.argtypes = [C.c_int64]
    lib.minima_fraction.argtypes = [P(ffg_graph), vp, vp, vp, vp, sz, vp]
    lib.walk_workspace_bytes.restype = sz
    lib.walk_workspace_bytes.argtypes = []
    lib.walk_simulate.argtypes = [P(ffg_graph), C.c_uint64, C.c_int64, vp, vp, sz,
                                  P(C.c_int64), vp]
    lib.dag_workspace_bytes.restype = sz
    lib.dag_workspace_bytes.argtypes = [C.c_int64]
    lib.dag_solve.argtypes = [P(ffg_graph), C.c_double, C.c_int, vp, vp, sz, P(C.c_int32), vp]
    lib.ffg_build_batch_workspace_bytes.restype = sz
    lib.ffg_build_batch_workspace_bytes.argtypes = [P(ffg_build_job), i32]
    lib.ffg_build_batch_count.argtypes = [P(ffg_build_job), i32, vp, sz, P(ffg_build_batch), vp]
    lib.ffg_build_batch_fill.argtypes = [P(ffg_build_job), i32, P(ffg_build_batch), vp]
    lib.ffg_build_batch_rerun.argtypes = [P(ffg_build_batch), vp]
    lib.ffg_build_batch_query.argtypes = [P(ffg_build_batch), vp, vp]
    lib.pagerank_batch_plan_tuned.argtypes = [P(ffg_pr_job), i32, C.c_int, P(ffg_pr_tuning), vp,
                                              sz, P(ffg_pr_batch), vp]
    lib.pagerank_batch_run.argtypes = [P(ffg_pr_batch), vp]
    lib.pagerank_batch_prepare.argtypes = [P(ffg_pr_batch), vp]
    lib.pagerank_batch_solve.argtypes = [P(ffg_pr_batch), vp]
    lib.pagerank_batch_query.argtypes = [P(ffg_pr_batch), vp, vp, vp, vp]
    lib.pagerank_batch_times.argtypes = [P(ffg_pr_batch), vp, vp]
    lib.pagerank_rows_w_bytes.argtypes = [C.c_int]
    lib.pagerank_rows_w_bytes.restype = sz
    lib.pagerank_rows_workspace_bytes.argtypes = [P(ffg_graph), i64, i64, C.c_int]
    lib.pagerank_rows_workspace_bytes.restype = sz
    lib.pagerank_rows_prepare.argtypes = [P(ffg_graph), i64, i64, C.c_int, vp, sz, vp]
    lib.pagerank_rows_run.argtypes = [P(ffg_graph), i64, i64, C.c_int, P(ffg_rows_op), vp, sz,
                                      vp]
    lib.centrality_workspace_bytes.argtypes = [i32]
    lib.centrality_workspace_bytes.restype = sz
    lib.centrality_proportion.argtypes = [P(ffg_graph), vp, vp, C.c_int, vp, i32, vp, vp, sz, vp]
    lib.centrality_batch_workspace_bytes.argtypes = [i32, i32]
    lib.centrality_batch_workspace_bytes.restype = sz
    lib.centrality_batch.argtypes = [P(ffg_cp_job), i32, C.c_int, vp, i32, vp, vp, sz, vp]
    lib.centrality_batch_plan.argtypes = [P(ffg_cp_job), i32, C.c_int, vp, i32, vp, sz,
                                          P(ffg_cp_batch), vp]
    lib.centrality_batch_run.argtypes = [P(ffg_cp_batch), vp]
    lib.centrality_batch_query.argtypes = [P(ffg_cp_batch), vp, vp, vp]
    lib.ffg_batch_run.argtypes = [P(ffg_batch_desc), P(ffg_batch_out), vp]
    lib.ffg_status_str.argtypes = [C.c_int]
    lib.ffg_status_str.restype = C.c_char_p
    lib.ffg_last_error.argtypes = []
    lib.ffg_last_error.restype = C.c_char_p
    lib.ffg_launch_count.argtypes = []
    lib.ffg_launch_count.restype = C.c_uint64
    lib.ffg_checked_build.argtypes = []
    lib.ffg_checked_build.restype = C.c_int
    lib.ffg_checked_failures.argtypes = [P(C.c_uint64), C.c_int]
    lib.ffg_checked_failures.restype = C.c_uint64
    if path is None:
        _lib = lib
    return lib


# ---- same-name wrappers ----------------------------------------------------

def ffg_status_str(status: int) -> str:
    return load().ffg_status_str(int(status)).decode()


def ffg_last_error() -> str:
    return load().ffg_last_error().decode()


def ffg_launch_count() -> int:
    return int(load().ffg_launch_count())


def ffg_checked_build() -> bool:
    return bool(load().ffg_checked_build())


def ffg_checked_failures(reset: bool = False) -> tuple[int, int]:
    """(failed checks since the last reset, site code of the first one)."""
    first = C.c_uint64(0)
    n = load().ffg_checked_failures(C.byref(first), int(bool(reset)))
    return int(n), int(first.value)


def ffg_workspace_bytes(space: "Space", nbh: int) -> int:
    return int(load().ffg_workspace_bytes(C.byref(space.c), int(nbh)))


def ffg_build_count(space, fitness_raw: int, nbh: int, fail_thr: float, g: ffg_graph,
                    ws: int, ws_bytes: int, stream: int = 0) -> int:
    return int(load().ffg_build_count(C.byref(space.c), C.c_void_p(fitness_raw), int(nbh),
                                      float(fail_thr), C.byref(g), None, None, C.c_void_p(ws),
                                      int(ws_bytes), C.c_void_p(stream)))


def ffg_build_fill(space, fitness_raw: int, nbh: int, fail_thr: float, g: ffg_graph, ws: int,
                   ws_bytes: int, stream: int = 0) -> int:
    return int(load().ffg_build_fill(C.byref(space.c), C.c_void_p(fitness_raw), int(nbh),
                                     float(fail_thr), C.byref(g), C.c_void_p(ws), int(ws_bytes),
                                     C.c_void_p(stream)))


def pagerank_workspace_bytes(n_nodes: int, n_edges: int, prec: int) -> int:
    return int(load().pagerank_workspace_bytes(int(n_nodes), int(n_edges), int(prec)))


def pagerank_prepare(g: ffg_graph, prec: int, ws: int, ws_bytes: int, stream: int = 0) -> int:
    return int(load().pagerank_prepare(C.byref(g), int(prec), C.c_void_p(ws), int(ws_bytes),
                                       C.c_void_p(stream)))


def pagerank_solve(g: ffg_graph, damping: float, tol: float, max_iter: int, prec: int,
                   ranks: int, init: int, ws: int, ws_bytes: int, sync: bool = True,
                   stream: int = 0):
    """Returns (status, iters, residual); iters/residual are None when sync=False."""
    it, res = C.c_int32(-1), C.c_double(float("nan"))
    st = load().pagerank_solve(C.byref(g), float(damping), float(tol), int(max_iter), int(prec),
                               C.c_void_p(ranks), int(init), C.c_void_p(ws), int(ws_bytes),
                               C.byref(it) if sync else None, C.byref(res) if sync else None,
                               C.c_void_p(stream))
    return (int(st), int(it.value), float(res.value)) if sync else (int(st), None, None)


def pagerank_solve_static(g: ffg_graph, damping: float, tol: float, max_iter: int, prec: int,
                          ranks: int, init: int = 0, stream: int = 0):
    """PageRank without a workspace (scratch in the library's static device
    array, 8 MiB).  For callers that cannot allocate device memory.
    Returns (status, iters, residual)."""
    it, res = C.c_int32(-1), C.c_double(float("nan"))
    st = load().pagerank_solve_static(C.byref(g), float(damping), float(tol), int(max_iter),
                                      int(prec), C.c_void_p(ranks), int(init), C.byref(it),
                                      C.byref(res), C.c_void_p(stream))
    return int(st), int(it.value), float(res.value)


def pagerank_batch_workspace_bytes(jobs, prec: int) -> int:
    return int(load().pagerank_batch_workspace_bytes(jobs, len(jobs), int(prec)))


def pagerank_batch_plan(jobs, prec: int, ws: int, ws_bytes: int, plan: "ffg_pr_batch",
                        stream: int = 0) -> int:
    return int(load().pagerank_batch_plan(jobs, len(jobs), int(prec), C.c_void_p(ws),
                                          int(ws_bytes), C.byref(plan), C.c_void_p(stream)))


def pagerank_batch_plan_tuned(jobs, prec: int, tuning, ws: int, ws_bytes: int,
                              plan: "ffg_pr_batch", stream: int = 0, job_cost=None) -> int:
    """``tuning``: (split, grain, max_blocks[, block_warps[, claim[, fp64_form[,
    min_tiles]]]]]); ``job_cost``: per-job costs replacing the cost model (or None)."""
    t = ffg_pr_tuning(float(tuning[0]), float(tuning[1]), int(tuning[2]),
                      int(tuning[3]) if len(tuning) > 3 else 0,
                      int(tuning[4]) if len(tuning) > 4 else 0,
                      int(tuning[5]) if len(tuning) > 5 else 0,
                      int(tuning[6]) if len(tuning) > 6 else 0)
    cost = None
    if job_cost is not None:
        cost = np.ascontiguousarray(job_cost, dtype=np.float64)
        if cost.shape != (len(jobs),):
            raise ValueError("job_cost needs one value per job")
        t.job_cost = cost.ctypes.data_as(C.POINTER(C.c_double))
    return int(load().pagerank_batch_plan_tuned(jobs, len(jobs), int(prec), C.byref(t),
                                                C.c_void_p(ws), int(ws_bytes), C.byref(plan),
                                                C.c_void_p(stream)))


def pagerank_batch_run(plan: "ffg_pr_batch", stream: int = 0) -> int:
    return int(load().pagerank_batch_run(C.byref(plan), C.c_void_p(stream)))


def pagerank_batch_prepare(plan: "ffg_pr_batch", stream: int = 0) -> int:
    return int(load().pagerank_batch_prepare(C.byref(plan), C.c_void_p(stream)))


def pagerank_batch_solve(plan: "ffg_pr_batch", stream: int = 0) -> int:
    return int(load().pagerank_batch_solve(C.byref(plan), C.c_void_p(stream)))


def pagerank_batch_query(plan: "ffg_pr_batch", stream: int = 0):
    """Returns (status, iters[n_jobs], residual[n_jobs], status[n_jobs])."""
    n = plan.n_jobs
    it = np.zeros(n, dtype=np.int32)
    res = np.zeros(n, dtype=np.float64)
    st = np.zeros(n, dtype=np.int32)
    s = load().pagerank_batch_query(C.byref(plan), C.c_void_p(it.ctypes.data),
                                    C.c_void_p(res.ctypes.data), C.c_void_p(st.ctypes.data),
                                    C.c_void_p(stream))
    return int(s), it, res, st


def pagerank_batch_times(plan: "ffg_pr_batch", stream: int = 0):
    """Returns (status, block-seconds[n_jobs]) of the last run."""
    out = np.zeros(plan.n_jobs, dtype=np.float64)
    s = load().pagerank_batch_times(C.byref(plan), C.c_void_p(out.ctypes.data),
                                    C.c_void_p(stream))
    return int(s), out


def pagerank_rows_w_bytes(prec: int) -> int:
    return int(load().pagerank_rows_w_bytes(int(prec)))


def pagerank_rows_workspace_bytes(g: "ffg_graph", row0: int, row1: int, prec: int) -> int:
    return int(load().pagerank_rows_workspace_bytes(C.byref(g), int(row0), int(row1), int(prec)))


def pagerank_rows_prepare(g: "ffg_graph", row0: int, row1: int, prec: int, ws: int,
                          ws_bytes: int, stream: int = 0) -> int:
    return int(load().pagerank_rows_prepare(C.byref(g), int(row0), int(row1), int(prec),
                                            C.c_void_p(ws), int(ws_bytes), C.c_void_p(stream)))


def pagerank_rows_run(g: "ffg_graph", row0: int, row1: int, prec: int, op: "ffg_rows_op",
                      ws: int, ws_bytes: int, stream: int = 0) -> int:
    return int(load().pagerank_rows_run(C.byref(g), int(row0), int(row1), int(prec),
                                        C.byref(op), C.c_void_p(ws), int(ws_bytes),
                                        C.c_void_p(stream)))


def pagerank_query(ws: int, stream: int = 0):
    it, res = C.c_int32(-1), C.c_double(float("nan"))
    st = load().pagerank_query(C.c_void_p(ws), C.byref(it), C.byref(res), C.c_void_p(stream))
    return int(st), int(it.value), float(res.value)


def centrality_workspace_bytes(n_p: int) -> int:
    return int(load().centrality_workspace_bytes(int(n_p)))


def centrality_proportion(g: ffg_graph, fitness_raw: int, ranks: int, prec: int, p, cp_out,
                          ws: int, ws_bytes: int, stream: int = 0) -> int:
    pv = np.ascontiguousarray(p, dtype=np.float64)
    assert cp_out.dtype == np.float64 and cp_out.flags.c_contiguous and len(cp_out) >= len(pv)
    return int(load().centrality_proportion(
        C.byref(g), C.c_void_p(fitness_raw), C.c_void_p(ranks), int(prec),
        C.c_void_p(pv.ctypes.data), len(pv), C.c_void_p(cp_out.ctypes.data), C.c_void_p(ws),
        int(ws_bytes), C.c_void_p(stream)))


# ---- tensor helpers ----------------------------------------------------------

class Space:
    """A search space in the C layout (host arrays kept alive here).

    ``values``: list of integer value lists (one per parameter);
    ``constraints``: list of (kind, params_a, params_b, bound) with kind one of
    'prod_le', 'prod_ge', 'divides', 'prod_le_prod' (or the integer codes)
    and params_* iterables of parameter indices.
    """

    def __init__(self, values, constraints=()):
        self.radix = np.ascontiguousarray([len(v) for v in values], dtype=np.int32)
        flat = [int(x) for v in values for x in v]
        self.values = np.ascontiguousarray(flat if flat else [0], dtype=np.int64)
        self.constraints = (ffg_constraint * max(len(constraints), 1))()
        for k, (kind, pa, pb, bound) in enumerate(constraints):
            ma = mb = 0
            for i in pa:
                if ma >> i & 1:
                    raise ValueError("a parameter appears twice in one product")
                ma |= 1 << int(i)
            for i in pb:
                if mb >> i & 1:
                    raise ValueError("a parameter appears twice in one product")
                mb |= 1 << int(i)
            c = self.constraints[k]
            c.kind = _KIND[kind] if isinstance(kind, str) else int(kind)
            c.mask_a, c.mask_b, c.reserved, c.bound = ma, mb, 0, int(bound)
        self.c = ffg_space(len(values), self.radix.ctypes.data_as(C.POINTER(C.c_int32)),
                           self.values.ctypes.data_as(C.POINTER(C.c_int64)), len(constraints),
                           C.cast(self.constraints, C.POINTER(ffg_constraint)))
        self.n_raw = int(np.prod(self.radix.astype(np.int64))) if len(values) else 0

    @classmethod
    def from_spec(cls, spec) -> "Space":
        """From any object with ``values`` and ``clauses`` (kind, a, b, bound)."""
        return cls(spec.values, [(cl.kind, cl.a, cl.b, cl.bound) for cl in spec.clauses])


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Graph:
    """An FFG in device tensors plus its ``ffg_graph`` struct."""

    def __init__(self, n_raw, n_nodes, n_edges, n_minima, f_opt, device):
        torch = _torch()
        self.out_ptr = torch.empty(n_nodes + 1, dtype=torch.int64, device=device)
        self.in_ptr = torch.empty(n_nodes + 1, dtype=torch.int64, device=device)
        self.out_idx = torch.empty(max(n_edges, 1), dtype=torch.int32, device=device)
        self.in_idx = torch.empty(max(n_edges, 1), dtype=torch.int32, device=device)
        self.outdeg = torch.empty(n_nodes, dtype=torch.int32, device=device)
        self.node_raw = torch.empty(n_nodes, dtype=torch.int64, device=device)
        self.is_min = torch.empty(n_nodes, dtype=torch.uint8, device=device)
        self.c = ffg_graph(n_raw, n_nodes, n_edges, n_minima, self.out_ptr.data_ptr(),
                           self.out_idx.data_ptr(), self.in_ptr.data_ptr(),
                           self.in_idx.data_ptr(), self.outdeg.data_ptr(),
                           self.node_raw.data_ptr(), self.is_min.data_ptr(), f_opt)

    n_raw = property(lambda self: int(self.c.n_raw))
    n_nodes = property(lambda self: int(self.c.n_nodes))
    n_edges = property(lambda self: int(self.c.n_edges))
    n_minima = property(lambda self: int(self.c.n_minima))
    f_opt = property(lambda self: float(self.c.f_opt))

    _ARRAYS = ("out_ptr", "in_ptr", "out_idx", "in_idx", "outdeg", "node_raw", "is_min")

    def save(self, path):
        """Checkpoint the graph as a CSR ``.npz`` (host copies of every array and
        the sizes); ``load_graph`` restores it."""
        e = self.n_edges
        arrays = {}
        for name in self._ARRAYS:
            t = getattr(self, name)
            arrays[name] = (t[:e] if name in ("out_idx", "in_idx") else t).cpu().numpy()
        np.savez(path, n_raw=self.n_raw, n_nodes=self.n_nodes, n_edges=e,
                 n_minima=self.n_minima, f_opt=self.f_opt, nbh=getattr(self, "nbh", -1),
                 **arrays)


def load_graph(path, device="cuda") -> Graph:
    """A graph saved by ``Graph.save``, in new tensors on ``device``."""
    torch = _torch()
    with np.load(path) as z:
        g = Graph(int(z["n_raw"]), int(z["n_nodes"]), int(z["n_edges"]), int(z["n_minima"]),
                  float(z["f_opt"]), device)
        for name in Graph._ARRAYS:
            src = torch.from_numpy(np.ascontiguousarray(z[name]))
            dst = getattr(g, name)
            if name in ("out_idx", "in_idx"):
                dst = dst[:src.numel()]
            if dst.shape != src.shape or dst.dtype != src.dtype:
                raise ValueError(f"{path}: array {name} has the wrong shape or type")
            dst.copy_(src)
        if int(z["nbh"]) >= 0:
            g.nbh = int(z["nbh"])
    return g


def _check(st, where, ok=(FFG_OK,)):
    if st not in ok:
        raise FFGError(st, where)
    return st


def workspace(nbytes: int, device="cuda"):
    torch = _torch()
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def build_graph(space: Space, fitness, nbh: int = HAMMING, fail_thr: float = 1e10, ws=None,
                stream=None) -> Graph:
    """Count, allocate, fill.  ``fitness``: CUDA float64 tensor of n_raw values."""
    torch = _torch()
    if not (fitness.is_cuda and fitness.dtype == torch.float64 and fitness.is_contiguous()):
        raise ValueError("fitness must be a contiguous CUDA float64 tensor")
    sh = _stream_handle(stream)
    need = ffg_workspace_bytes(space, nbh)
    if need == 0:
        raise FFGError(FFG_ERR_INVALID_ARG, "ffg_workspace_bytes")
    if ws is None or ws.numel() < need:
        ws = workspace(need, fitness.device)
    g0 = ffg_graph()
    _check(ffg_build_count(space, fitness.data_ptr(), nbh, fail_thr, g0, ws.data_ptr(), need, sh),
           "ffg_build_count")
    g = Graph(g0.n_raw, g0.n_nodes, g0.n_edges, g0.n_minima, g0.f_opt, fitness.device)
    _check(ffg_build_fill(space, fitness.data_ptr(), nbh, fail_thr, g.c, ws.data_ptr(), need, sh),
           "ffg_build_fill")
    g.nbh = nbh
    return g


DAG_VALUES, DAG_PAGERANK, DAG_ABSORB = 0, 1, 2


def dag_workspace_bytes(n_nodes: int) -> int:
    return int(load().dag_workspace_bytes(int(n_nodes)))


def dag_solve(g: "ffg_graph", damping: float, mode: int, ranks: int, ws: int, ws_bytes: int,
              stream: int = 0):
    """Returns (status, levels)."""
    lv = C.c_int32(0)
    s = load().dag_solve(C.byref(g), float(damping), int(mode), C.c_void_p(ranks),
                         C.c_void_p(ws), int(ws_bytes), C.byref(lv), C.c_void_p(stream))
    return int(s), int(lv.value)


def dag(g: "Graph", damping: float = 0.85, mode: int = DAG_PAGERANK, stream=None):
    """Exact solve on the DAG; returns (float64 tensor, levels)."""
    torch = _torch()
    dev = g.out_ptr.device
    out = torch.empty(g.n_nodes, dtype=torch.float64, device=dev)
    need = dag_workspace_bytes(g.n_nodes)
    ws = workspace(need, dev)
    st, lv = dag_solve(g.c, damping, mode, out.data_ptr(), ws.data_ptr(), need,
                       _stream_handle(stream))
    _check(st, "dag_solve")
    return out, lv


def minima_fraction(g: "Graph", fitness, stream=None):
    """(f_opt / f(x) of every local minimum, node ids), ascending node order."""
    torch = _torch()
    dev = g.out_ptr.device
    frac = torch.empty(max(g.n_minima, 1), dtype=torch.float64, device=dev)
    node = torch.empty(max(g.n_minima, 1), dtype=torch.int64, device=dev)
    need = int(load().minima_workspace_bytes(g.n_nodes))
    ws = workspace(need, dev)
    _check(int(load().minima_fraction(C.byref(g.c), C.c_void_p(fitness.data_ptr()),
                                      C.c_void_p(frac.data_ptr()), C.c_void_p(node.data_ptr()),
                                      C.c_void_p(ws.data_ptr()), need,
                                      C.c_void_p(_stream_handle(stream)))), "minima_fraction")
    return frac[:g.n_minima], node[:g.n_minima]


def walk_simulate(g: "ffg_graph", seed: int, n_walks: int, counts: int, ws: int,
                  ws_bytes: int, stream: int = 0):
    """Returns (status, steps)."""
    steps = C.c_int64(0)
    s = load().walk_simulate(C.byref(g), int(seed) & 0xFFFFFFFFFFFFFFFF, int(n_walks),
                             C.c_void_p(counts), C.c_void_p(ws), int(ws_bytes),
                             C.byref(steps), C.c_void_p(stream))
    return int(s), int(steps.value)


def walks(g: "Graph", seed: int, n_walks: int, stream=None):
    """Improving-walk arrival counts (int64 tensor) and the number of moves."""
    torch = _torch()
    dev = g.out_ptr.device
    counts = torch.empty(g.n_nodes, dtype=torch.int64, device=dev)
    ws = workspace(int(load().walk_workspace_bytes()), dev)
    st, steps = walk_simulate(g.c, seed, n_walks, counts.data_ptr(), ws.data_ptr(), ws.numel(),
                              _stream_handle(stream))
    _check(st, "walk_simulate")
    return counts, steps


class BuildBatch:
    """FFGs of many spaces built together: ``specs`` is a list of (Space,
    fitness CUDA float64 tensor, nbh).  Counts all (one synchronisation),
    allocates every Graph, fills all.  ``rerun()`` repeats the whole build
    with launches only (capturable); ``query()`` returns the per-job status
    array."""

    def __init__(self, specs, fail_thr: float = 1e10, stream=None):
        torch = _torch()
        self.specs = list(specs)
        n = len(self.specs)
        self.jobs = (ffg_build_job * n)()
        self._g0 = [ffg_graph() for _ in range(n)]
        for k, (sp, fit, nbh) in enumerate(self.specs):
            if not (fit.is_cuda and fit.dtype == torch.float64 and fit.is_contiguous()):
                raise ValueError("fitness must be a contiguous CUDA float64 tensor")
            self.jobs[k].space = C.pointer(sp.c)
            self.jobs[k].fitness_raw = fit.data_ptr()
            self.jobs[k].nbh = int(nbh)
            self.jobs[k].fail_thr = float(fail_thr)
            self.jobs[k].g = C.pointer(self._g0[k])
        need = int(load().ffg_build_batch_workspace_bytes(self.jobs, n))
        if need == 0:
            raise FFGError(FFG_ERR_INVALID_ARG, "ffg_build_batch_workspace_bytes")
        dev = self.specs[0][1].device
        self.ws = workspace(need, dev)
        self.plan = ffg_build_batch()
        sh = _stream_handle(stream)
        _check(int(load().ffg_build_batch_count(self.jobs, n, C.c_void_p(self.ws.data_ptr()),
                                                need, C.byref(self.plan), C.c_void_p(sh))),
               "ffg_build_batch_count")
        self.graphs = []
        for k, g0 in enumerate(self._g0):
            g = Graph(g0.n_raw, g0.n_nodes, g0.n_edges, g0.n_minima, g0.f_opt, dev)
            g.nbh = self.specs[k][2]
            self.graphs.append(g)
            self.jobs[k].g = C.pointer(g.c)
        _check(int(load().ffg_build_batch_fill(self.jobs, n, C.byref(self.plan), C.c_void_p(sh))),
               "ffg_build_batch_fill")

    def rerun(self, stream=None):
        _check(int(load().ffg_build_batch_rerun(C.byref(self.plan),
                                                C.c_void_p(_stream_handle(stream)))),
               "ffg_build_batch_rerun")

    def query(self, stream=None):
        st = np.zeros(len(self.specs), dtype=np.int32)
        s = int(load().ffg_build_batch_query(C.byref(self.plan), C.c_void_p(st.ctypes.data),
                                             C.c_void_p(_stream_handle(stream))))
        return s, st


def pagerank(g: Graph, damping: float = 0.85, tol: float = 1e-12, max_iter: int = 10000,
             prec: int = F64, init=None, ws=None, out=None, stream=None, prepared=False):
    """Returns (ranks tensor, iters, residual, converged).  ``prepared``: the
    workspace ``ws`` already holds this graph's layout (pagerank_prepare)."""
    torch = _torch()
    dt = torch.float64 if prec == F64 else torch.float32
    dev = g.out_ptr.device
    ranks = out if out is not None else torch.empty(g.n_nodes, dtype=dt, device=dev)
    if init is not None:
        ranks.copy_(init)
    need = pagerank_workspace_bytes(g.n_nodes, g.n_edges, prec)
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    flags = (INIT_RANKS if init is not None else 0) | (INIT_LAYOUT if prepared else 0)
    st, it, res = pagerank_solve(g.c, damping, tol, max_iter, prec, ranks.data_ptr(), flags,
                                 ws.data_ptr(), need, True, _stream_handle(stream))
    _check(st, "pagerank_solve", ok=(FFG_OK, FFG_ERR_NOT_CONVERGED))
    return ranks, it, res, st == FFG_OK


def centrality_batch_workspace_bytes(n_jobs: int, n_p: int) -> int:
    return int(load().centrality_batch_workspace_bytes(int(n_jobs), int(n_p)))


def centrality_batch(jobs, prec: int, p, cp_out, ws: int, ws_bytes: int, stream: int = 0) -> int:
    pv = np.ascontiguousarray(p, dtype=np.float64)
    assert cp_out.dtype == np.float64 and cp_out.size >= len(jobs) * len(pv)
    return int(load().centrality_batch(jobs, len(jobs), int(prec), C.c_void_p(pv.ctypes.data),
                                       len(pv), C.c_void_p(cp_out.ctypes.data), C.c_void_p(ws),
                                       int(ws_bytes), C.c_void_p(stream)))


def ffg_batch_run(desc: "ffg_batch_desc", out: "ffg_batch_out | None", stream: int = 0) -> int:
    return int(load().ffg_batch_run(C.byref(desc), C.byref(out) if out is not None else None,
                                    C.c_void_p(stream)))


def centrality_many(specs, p, stream=None) -> np.ndarray:
    """C_p of many graphs at once; ``specs``: list of (Graph, fitness, ranks)."""
    torch = _torch()
    jobs = (ffg_cp_job * len(specs))()
    for k, (g, fit, x) in enumerate(specs):
        jobs[k].g = C.pointer(g.c)
        jobs[k].fitness_raw = fit.data_ptr()
        jobs[k].ranks = x.data_ptr()
    prec = F64 if specs[0][2].dtype == torch.float64 else F32
    need = centrality_batch_workspace_bytes(len(specs), len(p))
    ws = workspace(need, specs[0][2].device)
    out = np.zeros((len(specs), len(p)), dtype=np.float64)
    _check(centrality_batch(jobs, prec, p, out, ws.data_ptr(), need, _stream_handle(stream)),
           "centrality_batch")
    return out


def centrality_batch_plan(jobs, prec: int, p, ws: int, ws_bytes: int, plan: "ffg_cp_batch",
                          stream: int = 0) -> int:
    pv = np.ascontiguousarray(p, dtype=np.float64)
    return int(load().centrality_batch_plan(jobs, len(jobs), int(prec), C.c_void_p(pv.ctypes.data),
                                            len(pv), C.c_void_p(ws), int(ws_bytes),
                                            C.byref(plan), C.c_void_p(stream)))


def centrality_batch_run(plan: "ffg_cp_batch", stream: int = 0) -> int:
    return int(load().centrality_batch_run(C.byref(plan), C.c_void_p(stream)))


def centrality_batch_query(plan: "ffg_cp_batch", stream: int = 0):
    """Returns (status, cp (n_jobs x n_p), per-job statuses)."""
    cp = np.full((plan.n_jobs, plan.n_p), np.nan)
    st = np.zeros(plan.n_jobs, dtype=np.int32)
    s = int(load().centrality_batch_query(C.byref(plan), C.c_void_p(cp.ctypes.data),
                                          C.c_void_p(st.ctypes.data), C.c_void_p(stream)))
    return s, cp, st


class CentralityBatch:
    """C_p of many graphs, planned once (``centrality_batch_plan``); ``run()``
    only enqueues kernels (capturable), the results stay on the device in
    ``cp`` / ``status`` until ``query()``.  ``specs``: list of (Graph,
    fitness, ranks)."""

    def __init__(self, specs, p, stream=None):
        torch = _torch()
        self.jobs = (ffg_cp_job * len(specs))()
        for k, (g, fit, x) in enumerate(specs):
            self.jobs[k].g = C.pointer(g.c)
            self.jobs[k].fitness_raw = fit.data_ptr()
            self.jobs[k].ranks = x.data_ptr()
        self.prec = F64 if specs[0][2].dtype == torch.float64 else F32
        self.p = np.ascontiguousarray(p, dtype=np.float64)
        need = centrality_batch_workspace_bytes(len(specs), len(self.p))
        self.ws = workspace(need, specs[0][2].device)
        self.plan = ffg_cp_batch()
        _check(centrality_batch_plan(self.jobs, self.prec, self.p, self.ws.data_ptr(), need,
                                     self.plan, _stream_handle(stream)), "centrality_batch_plan")

    def run(self, stream=None):
        _check(centrality_batch_run(self.plan, _stream_handle(stream)), "centrality_batch_run")

    def query(self, stream=None):
        st, cp, sts = centrality_batch_query(self.plan, _stream_handle(stream))
        _check(st, "centrality_batch_query", ok=(FFG_OK, FFG_ERR_EMPTY))
        return cp, sts


class PageRankBatch:
    """Many PageRank solves in one persistent launch (``pagerank_batch_*``).

    ``specs``: list of (Graph, damping).  Holds the job array, the workspace,
    the plan and the output tensors; ``run()`` only enqueues kernels, so it can
    be captured in a CUDA graph; ``query()`` synchronises and returns the
    per-job iterations, residuals and statuses."""

    def __init__(self, specs, prec: int = F32, tol: float = 1e-12, max_iter: int = 10000,
                 stream=None):
        torch = _torch()
        dt = torch.float64 if prec == F64 else torch.float32
        self.graphs = [g for g, _ in specs]
        self.ranks = [torch.empty(g.n_nodes, dtype=dt, device=g.out_ptr.device) for g in self.graphs]
        self.jobs = (ffg_pr_job * len(specs))()
        for k, (g, alpha) in enumerate(specs):
            self.jobs[k].g = C.pointer(g.c)
            self.jobs[k].damping = float(alpha)
            self.jobs[k].tol = float(tol)
            self.jobs[k].max_iter = int(max_iter)
            self.jobs[k].init = 0
            self.jobs[k].ranks = self.ranks[k].data_ptr()
        self.prec = prec
        need = pagerank_batch_workspace_bytes(self.jobs, prec)
        if need == 0:
            raise FFGError(FFG_ERR_INVALID_ARG, "pagerank_batch_workspace_bytes")
        self.ws = workspace(need, self.graphs[0].out_ptr.device)
        self.need = need
        self.plan = ffg_pr_batch()
        self.tuning = (0.05, 0.005, 0, 0, 0)   # pagerank_batch_plan's defaults
        self.job_cost = None
        _check(pagerank_batch_plan(self.jobs, prec, self.ws.data_ptr(), need, self.plan,
                                   _stream_handle(stream)), "pagerank_batch_plan")

    def replan(self, tuning, stream=None, job_cost=None):
        """Re-plan into the same workspace with (split, grain, max_blocks[, block_warps[,
        claim[, fp64_form[, min_tiles]]]]), and per-job costs in place of the model if
        given."""
        _check(pagerank_batch_plan_tuned(self.jobs, self.prec, tuning, self.ws.data_ptr(),
                                         self.need, self.plan, _stream_handle(stream),
                                         job_cost=job_cost),
               "pagerank_batch_plan_tuned")
        self.tuning = tuple(tuning)
        self.job_cost = None if job_cost is None else np.array(job_cost, dtype=np.float64)

    def run(self, stream=None):
        _check(pagerank_batch_run(self.plan, _stream_handle(stream)), "pagerank_batch_run")

    def prepare(self, stream=None):
        """The edge layout of every graph alone (``pagerank_batch_prepare``)."""
        _check(pagerank_batch_prepare(self.plan, _stream_handle(stream)),
               "pagerank_batch_prepare")

    def solve(self, stream=None):
        """The persistent solve alone, on the current layout (``pagerank_batch_solve``)."""
        _check(pagerank_batch_solve(self.plan, _stream_handle(stream)), "pagerank_batch_solve")

    def query(self, stream=None):
        st, it, res, sts = pagerank_batch_query(self.plan, _stream_handle(stream))
        _check(st, "pagerank_batch_query", ok=(FFG_OK, FFG_ERR_NOT_CONVERGED))
        return it, res, sts

    def times(self, stream=None):
        """Per-job block-seconds of the last run (``pagerank_batch_times``)."""
        st, t = pagerank_batch_times(self.plan, _stream_handle(stream))
        _check(st, "pagerank_batch_times")
        return t


def centrality(g: Graph, fitness, ranks, p, ws=None, stream=None) -> np.ndarray:
    torch = _torch()
    prec = F64 if ranks.dtype == torch.float64 else F32
    need = centrality_workspace_bytes(len(p))
    if ws is None or ws.numel() < need:
        ws = workspace(need, ranks.device)
    out = np.zeros(len(p), dtype=np.float64)
    _check(centrality_proportion(g.c, fitness.data_ptr(), ranks.data_ptr(), prec, p, out,
                                 ws.data_ptr(), need, _stream_handle(stream)),
           "centrality_proportion")
    return out


class SpaceBatch:
    """A whole batch per call (``ffg_batch_run``): ``solves`` is a
    PageRankBatch; ``builds`` the BuildBatch of its graphs (rebuilt on every
    run) or None; ``cp`` a CentralityBatch over the solves' graphs and ranks
    (or None).

    ``run(sync=False)`` only enqueues kernels (capturable in a CUDA graph);
    ``run()`` synchronises and returns (status, outputs)."""

    def __init__(self, solves, builds=None, cp=None):
        self.solves, self.builds, self.cp = solves, builds, cp
        self.desc = ffg_batch_desc()
        self.desc.pagerank = C.pointer(solves.plan)
        if builds is not None:
            self.desc.build = C.pointer(builds.plan)
        if cp is not None:
            self.desc.cp = C.pointer(cp.plan)

    def run(self, sync: bool = True, stream=None):
        sh = _stream_handle(stream)
        if not sync:
            _check(ffg_batch_run(self.desc, None, sh), "ffg_batch_run")
            return None
        n = self.solves.plan.n_jobs
        res = {"iters": np.zeros(n, np.int32), "residual": np.zeros(n, np.float64),
               "pr_status": np.zeros(n, np.int32)}
        out = ffg_batch_out()
        out.iters = res["iters"].ctypes.data
        out.residual = res["residual"].ctypes.data
        out.pr_status = res["pr_status"].ctypes.data
        if self.builds is not None:
            res["build_status"] = np.zeros(self.builds.plan.n_jobs, np.int32)
            out.build_status = res["build_status"].ctypes.data
        if self.cp is not None:
            res["cp"] = np.full((self.cp.plan.n_jobs, self.cp.plan.n_p), np.nan)
            out.cp = res["cp"].ctypes.data
        st = ffg_batch_run(self.desc, out, sh)
        return st, res
