"""The C-ABI library loads, exports every function include/ffg.h declares, and
rejects bad arguments on the host (no GPU needed: argument errors are found
before any CUDA call)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import ffg_inputs as fi
import paper_2210_01465_gb300 as ffg

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "ffg.h")


@pytest.fixture(scope="module")
def lib():
    ffg.build()
    return ffg.load()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(\w+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("defined",)))


def test_header_declares_entry_points():
    names = _declared_functions()
    assert set(names) == set(ffg.ENTRY_POINTS), names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_checked_build_exports_the_same_symbols(lib):
    """The bounds-checked variant (-DFFG_CHECKED) builds, exports the same
    entry points and says which build it is; with no kernel run it has
    recorded no failed check (reading its record needs the GPU, so only the
    flag is read here)."""
    path = ffg.build(checked=True)
    chk = C.CDLL(path)
    for name in _declared_functions():
        assert hasattr(chk, name), name
    chk.ffg_checked_build.restype = C.c_int
    assert chk.ffg_checked_build() == 1
    assert lib.ffg_checked_build() == 0
    assert not ffg.ffg_checked_build()


def test_status_strings(lib):
    for s in range(8):
        assert ffg.ffg_status_str(s) not in ("", "unknown status")
    assert ffg.ffg_status_str(99) == "unknown status"


def test_space_validation_on_host(lib):
    ok = ffg.Space.from_spec(fi.single_small())
    assert ffg.ffg_workspace_bytes(ok, ffg.HAMMING) > 0
    bad = [
        ffg.Space([[1, 2]] * 17),                                  # too many parameters
        ffg.Space([[1, 2], []]),                                   # empty list
        ffg.Space([[1, 2]], [("prod_le", (3,), (), 4)]),           # mask beyond n_params
        ffg.Space([list(range(2000))]),                            # too many values
        ffg.Space([list(range(1, 50))] * 6),                       # more than 2^31-1 points
        ffg.Space([[1 << 40, 2], [1 << 40, 3]], [("prod_le", (0, 1), (), 5)]),  # int64 overflow
    ]
    for sp in bad:
        assert ffg.ffg_workspace_bytes(sp, ffg.HAMMING) == 0


def test_argument_errors_before_cuda(lib):
    sp = ffg.Space.from_spec(fi.single_small())
    g = ffg.ffg_graph()
    # NULL fitness / workspace
    assert ffg.ffg_build_count(sp, 0, ffg.HAMMING, 1e10, g, 0, 0) == ffg.FFG_ERR_INVALID_ARG
    # unknown neighbourhood
    assert ffg.ffg_build_count(sp, 256, 7, 1e10, g, 256, 1 << 30) == ffg.FFG_ERR_INVALID_ARG
    # misaligned workspace
    assert ffg.ffg_build_count(sp, 256, 0, 1e10, g, 258, 1 << 30) == ffg.FFG_ERR_INVALID_ARG
    # workspace too small
    assert ffg.ffg_build_count(sp, 256, 0, 1e10, g, 256, 16) == ffg.FFG_ERR_NO_MEMORY
    # overflow
    big = ffg.Space([list(range(1, 50))] * 6)
    assert ffg.ffg_build_count(big, 256, 0, 1e10, g, 256, 1 << 30) == ffg.FFG_ERR_OVERFLOW
    # fill without a count
    assert ffg.ffg_build_fill(sp, 256, 0, 1e10, g, 256, 1 << 30) == ffg.FFG_ERR_INVALID_ARG
    # pagerank: empty graph, bad damping, bad precision
    g.n_nodes, g.n_edges, g.in_ptr, g.in_idx, g.outdeg = 10, 5, 256, 256, 256
    e = ffg.ffg_graph()
    assert ffg.pagerank_solve(e, 0.85, 1e-9, 10, 0, 256, 0, 256, 1 << 20)[0] == 1
    for damping in (0.0, 1.0, -0.5, float("nan")):
        assert ffg.pagerank_solve(g, damping, 1e-9, 10, 0, 256, 0, 256, 1 << 20)[0] == 1
    assert ffg.pagerank_solve(g, 0.85, 1e-9, 0, 0, 256, 0, 256, 1 << 20)[0] == 1
    assert ffg.pagerank_solve(g, 0.85, 1e-9, ffg.MAX_ITER + 1, 0, 256, 0, 256, 1 << 20)[0] == 1
    assert "max_iter" in ffg.ffg_last_error()
    # the entry point without a workspace refuses unknown init flags up front
    assert ffg.pagerank_solve_static(g, 0.85, 1e-9, 10, 0, 256, 4, 0)[0] == 1
    assert "init" in ffg.ffg_last_error()
    assert ffg.pagerank_solve(g, 0.85, 1e-9, 10, 5, 256, 0, 256, 1 << 20)[0] == 1
    assert ffg.pagerank_solve(g, 0.85, 1e-9, 10, 0, 256, 0, 256, 8)[0] == ffg.FFG_ERR_NO_MEMORY
    assert ffg.pagerank_solve(g, 0.85, 1e-9, 10, 0, 256, 4, 256, 1 << 30)[0] == 1
    assert ffg.pagerank_prepare(e, 0, 256, 1 << 20) == 1
    assert ffg.pagerank_prepare(g, 0, 258, 1 << 20) == 1
    # centrality: n_p out of range, negative p
    g.is_min, g.node_raw, g.n_minima = 256, 256, 1
    out = np.zeros(40)
    assert ffg.centrality_proportion(g, 256, 256, 0, [], out, 256, 1 << 20) == 1
    assert ffg.centrality_proportion(g, 256, 256, 0, [0.1] * 33, out, 256, 1 << 20) == 1
    assert ffg.centrality_proportion(g, 256, 256, 0, [-0.1], out, 256, 1 << 20) == 1
    assert ffg.centrality_proportion(g, 256, 256, 0, [np.inf], out, 256, 1 << 20) == 1
    g.n_minima = 0
    assert ffg.centrality_proportion(g, 256, 256, 0, [0.1], out, 256, 1 << 20) == \
        ffg.FFG_ERR_EMPTY
    assert "workspace" in ffg.ffg_last_error() or ffg.ffg_last_error() != ""


def test_workspace_sizes_monotone(lib):
    small = ffg.Space.from_spec(fi.single_small())
    large = ffg.Space.from_spec(fi.single_large())
    assert ffg.ffg_workspace_bytes(large, 0) > ffg.ffg_workspace_bytes(small, 0)
    assert ffg.pagerank_workspace_bytes(10**6, 10**7, ffg.F64) > ffg.pagerank_workspace_bytes(10**6, 10**7, ffg.F32)
    assert ffg.centrality_workspace_bytes(5) > 0


def test_product_path_has_no_oracle_import():
    """The library package neither imports nor names the oracle."""
    pkg = os.path.dirname(ffg.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(root, f)).read()
                assert "import oracle" not in src and "ffg_oracle" not in src, f


def test_batch_tuning_validated_on_host(lib):
    jobs = (ffg.ffg_pr_job * 1)()
    plan = ffg.ffg_pr_batch()
    for tuning in ((0.0, 1.0, 0), (1.0, -1.0, 0), (float("nan"), 1.0, 0), (1.0, 1.0, -2),
                   (1.0, 1.0, 0, 12), (1.0, 1.0, 0, 32), (1.0, 1.0, 0, 8, 2), (1.0, 1.0, 0, 8, 0, 3),
                   (1.0, 1.0, 0, 24, 1, 0, -1), (1.0, 1.0, 0, 24, 0, 0, (1 << 20) + 1)):
        assert ffg.pagerank_batch_plan_tuned(jobs, ffg.F32, tuning, 256, 1 << 20, plan) == \
            ffg.FFG_ERR_INVALID_ARG
        assert "tuning" in ffg.ffg_last_error()
    # measured job costs: positive and finite, checked before any planning
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        assert ffg.pagerank_batch_plan_tuned(jobs, ffg.F32, (1.0, 1.0, 0), 256, 1 << 20, plan,
                                             job_cost=[bad]) == ffg.FFG_ERR_INVALID_ARG
        assert "job_cost" in ffg.ffg_last_error()
    with pytest.raises(ValueError):
        ffg.pagerank_batch_plan_tuned(jobs, ffg.F32, (1.0, 1.0, 0), 256, 1 << 20, plan,
                                      job_cost=[1.0, 2.0])
    assert ffg.pagerank_batch_times(ffg.ffg_pr_batch())[0] == ffg.FFG_ERR_INVALID_ARG
    assert lib.pagerank_batch_times(None, None, None) == ffg.FFG_ERR_INVALID_ARG


def test_rows_validated_on_host(lib):
    """The row-range entry points refuse bad ranges, operations and dampings
    before any device access."""
    g = ffg.ffg_graph()
    g.n_nodes, g.n_edges = 100, 400
    g.in_ptr, g.in_idx, g.outdeg = 256, 256, 256
    assert ffg.pagerank_rows_w_bytes(ffg.F32) == 4 and ffg.pagerank_rows_w_bytes(ffg.F64) == 16
    assert ffg.pagerank_rows_w_bytes(7) == 0
    for r0, r1 in ((0, 0), (5, 4), (-1, 10), (90, 101)):
        assert ffg.pagerank_rows_workspace_bytes(g, r0, r1, ffg.F32) == 0
        assert ffg.pagerank_rows_prepare(g, r0, r1, ffg.F32, 256, 1 << 20) == \
            ffg.FFG_ERR_INVALID_ARG
        assert "rows" in ffg.ffg_last_error()
    before = lib.ffg_launch_count()
    sums = np.zeros(4, dtype=np.uint64)
    ctl = np.zeros(ffg.ROWS_CTL_BYTES, dtype=np.uint8)
    op = ffg.ffg_rows_op(ffg.ROWS_STEP, 1, 1.0, 0.0, 256, 256, None, sums.ctypes.data,
                         ctl.ctypes.data)
    assert ffg.pagerank_rows_run(g, 0, 50, ffg.F32, op, 256, 1 << 20) == ffg.FFG_ERR_INVALID_ARG
    assert "damping" in ffg.ffg_last_error()
    op.op = 9
    assert ffg.pagerank_rows_run(g, 0, 50, ffg.F32, op, 256, 1 << 20) == ffg.FFG_ERR_INVALID_ARG
    op.op = ffg.ROWS_WRITE
    assert ffg.pagerank_rows_run(g, 0, 50, ffg.F32, op, 256, 1 << 20) == ffg.FFG_ERR_INVALID_ARG
    op.op, op.max_iter = ffg.ROWS_ADVANCE, 0           # the stopping rule needs max_iter >= 1
    assert ffg.pagerank_rows_run(g, 0, 50, ffg.F32, op, 256, 1 << 20) == ffg.FFG_ERR_INVALID_ARG
    op.op, op.ctl = ffg.ROWS_START, None               # every operation needs the control record
    assert ffg.pagerank_rows_run(g, 0, 50, ffg.F32, op, 256, 1 << 20) == ffg.FFG_ERR_INVALID_ARG
    op.ctl = ctl.ctypes.data
    op.op, op.damping = ffg.ROWS_STEP, 0.85
    assert ffg.pagerank_rows_run(g, 0, 50, ffg.F32, op, 258, 1 << 20) == ffg.FFG_ERR_INVALID_ARG
    assert ffg.pagerank_rows_run(g, 0, 50, ffg.F32, op, 256, 64) == ffg.FFG_ERR_NO_MEMORY
    assert lib.ffg_launch_count() == before


def test_batch_run_validated_on_host(lib):
    """ffg_batch_run refuses a missing plan or incomplete C_p arguments
    before it launches anything."""
    before = lib.ffg_launch_count()
    assert lib.ffg_batch_run(None, None, None) == ffg.FFG_ERR_INVALID_ARG
    desc = ffg.ffg_batch_desc()
    assert ffg.ffg_batch_run(desc, None) == ffg.FFG_ERR_INVALID_ARG     # no PageRank plan
    plan = ffg.ffg_pr_batch()
    desc.pagerank = C.pointer(plan)
    assert ffg.ffg_batch_run(desc, None) == ffg.FFG_ERR_INVALID_ARG     # plan with no jobs
    plan.n_jobs = 1
    bplan = ffg.ffg_build_batch()
    desc.build = C.pointer(bplan)
    assert ffg.ffg_batch_run(desc, None) == ffg.FFG_ERR_INVALID_ARG     # empty build plan
    desc.build = None
    cp = np.zeros(4)
    out = ffg.ffg_batch_out()
    out.cp = cp.ctypes.data
    assert ffg.ffg_batch_run(desc, out) == ffg.FFG_ERR_INVALID_ARG      # C_p without a plan
    assert "C_p plan" in ffg.ffg_last_error()
    cplan = ffg.ffg_cp_batch()
    desc.cp = C.pointer(cplan)
    assert ffg.ffg_batch_run(desc, out) == ffg.FFG_ERR_INVALID_ARG      # empty C_p plan
    assert ffg.centrality_batch_run(cplan) == ffg.FFG_ERR_INVALID_ARG
    assert ffg.centrality_batch_query(cplan)[0] == ffg.FFG_ERR_INVALID_ARG
    jobs = (ffg.ffg_cp_job * 2)()
    assert ffg.centrality_batch_plan(jobs, ffg.F32, [0.05], 256, 1 << 20, cplan) == \
        ffg.FFG_ERR_INVALID_ARG                                          # jobs without graphs
    assert ffg.centrality_batch_plan(jobs, ffg.F32, [-0.05], 256, 1 << 20, cplan) == \
        ffg.FFG_ERR_INVALID_ARG
    assert ffg.centrality_batch_plan(jobs, ffg.F32, [0.05] * 33, 256, 1 << 20, cplan) == \
        ffg.FFG_ERR_INVALID_ARG
    assert lib.ffg_launch_count() == before


def test_batched_build_validated_on_host(lib):
    sp = ffg.Space.from_spec(fi.single_small())
    g = ffg.ffg_graph()
    jobs = (ffg.ffg_build_job * 2)()
    for j in jobs:
        j.space = C.pointer(sp.c)
        j.fitness_raw = 256
        j.nbh = ffg.HAMMING
        j.fail_thr = 1e10
        j.g = C.pointer(g)
    assert lib.ffg_build_batch_workspace_bytes(jobs, 2) > 2 * ffg.ffg_workspace_bytes(sp, 0) // 2
    assert lib.ffg_build_batch_workspace_bytes(jobs, 0) == 0
    plan = ffg.ffg_build_batch()
    jobs[1].nbh = 7
    assert lib.ffg_build_batch_workspace_bytes(jobs, 2) == 0
    assert lib.ffg_build_batch_count(jobs, 2, C.c_void_p(256), 1 << 30, C.byref(plan),
                                     None) == ffg.FFG_ERR_INVALID_ARG
    jobs[1].nbh = ffg.HAMMING
    jobs[1].fitness_raw = None
    assert lib.ffg_build_batch_count(jobs, 2, C.c_void_p(256), 1 << 30, C.byref(plan),
                                     None) == ffg.FFG_ERR_INVALID_ARG
    jobs[1].fitness_raw = 256
    assert lib.ffg_build_batch_count(jobs, 2, C.c_void_p(258), 1 << 30, C.byref(plan),
                                     None) == ffg.FFG_ERR_INVALID_ARG
    assert lib.ffg_build_batch_count(jobs, 2, C.c_void_p(256), 16, C.byref(plan),
                                     None) == ffg.FFG_ERR_NO_MEMORY
    assert lib.ffg_build_batch_rerun(C.byref(ffg.ffg_build_batch()), None) == \
        ffg.FFG_ERR_INVALID_ARG


def test_dag_solve_validated_on_host(lib):
    g = ffg.ffg_graph()
    g.n_nodes, g.n_edges = 10, 5
    g.in_ptr = g.out_ptr = g.in_idx = g.out_idx = g.outdeg = 256
    need = ffg.dag_workspace_bytes(10)
    assert need > 0
    assert ffg.dag_solve(ffg.ffg_graph(), 0.85, ffg.DAG_PAGERANK, 256, 256, need)[0] == 1
    for d, mode in ((1.0, ffg.DAG_PAGERANK), (0.0, ffg.DAG_PAGERANK), (0.85, ffg.DAG_ABSORB),
                    (1.5, ffg.DAG_VALUES), (-0.1, ffg.DAG_VALUES), (0.5, 7)):
        assert ffg.dag_solve(g, d, mode, 256, 256, need)[0] == ffg.FFG_ERR_INVALID_ARG
    assert ffg.dag_solve(g, 0.85, ffg.DAG_PAGERANK, 256, 258, need)[0] == ffg.FFG_ERR_INVALID_ARG
    assert ffg.dag_solve(g, 0.85, ffg.DAG_PAGERANK, 256, 256, 16)[0] == ffg.FFG_ERR_NO_MEMORY


def test_walk_simulate_validated_on_host(lib):
    g = ffg.ffg_graph()
    g.n_nodes, g.n_edges = 10, 5
    g.in_ptr = g.out_ptr = g.in_idx = g.out_idx = g.outdeg = 256
    assert lib.walk_workspace_bytes() == 256
    assert ffg.walk_simulate(ffg.ffg_graph(), 1, 10, 256, 256, 256)[0] == 1
    assert ffg.walk_simulate(g, 1, -1, 256, 256, 256)[0] == ffg.FFG_ERR_INVALID_ARG
    assert ffg.walk_simulate(g, 1, 10, 0, 256, 256)[0] == ffg.FFG_ERR_INVALID_ARG
    assert ffg.walk_simulate(g, 1, 10, 256, 258, 256)[0] == ffg.FFG_ERR_INVALID_ARG
    assert ffg.walk_simulate(g, 1, 10, 256, 256, 8)[0] == ffg.FFG_ERR_NO_MEMORY


def test_minima_fraction_validated_on_host(lib):
    g = ffg.ffg_graph()
    g.n_nodes, g.is_min, g.node_raw, g.n_minima = 10, 256, 256, 0
    need = lib.minima_workspace_bytes(10)
    assert need > 0
    args = (C.c_void_p(256), C.c_void_p(256), None, C.c_void_p(256), need, None)
    assert lib.minima_fraction(C.byref(g), *args) == ffg.FFG_ERR_EMPTY
    g.n_minima = 2
    assert lib.minima_fraction(C.byref(g), C.c_void_p(256), C.c_void_p(256), None,
                               C.c_void_p(258), need, None) == ffg.FFG_ERR_INVALID_ARG
    assert lib.minima_fraction(C.byref(g), C.c_void_p(256), C.c_void_p(256), None,
                               C.c_void_p(256), 8, None) == ffg.FFG_ERR_NO_MEMORY
