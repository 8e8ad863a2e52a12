"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Bars: FFG arrays and local-minimum sets bit-exact; FP64 ranks within L1 1e-9
of the oracle's exact solve; FP32 proportions of centrality within 1e-5
absolute (rank L1 error reported).  Sizes span several thread blocks and
ragged tails; the single-space workloads run at full size.
"""
import numpy as np
import pytest

import ffg_inputs as fi
import oracle

torch = pytest.importorskip("torch")
ffg = pytest.importorskip("paper_2210_01465_gb300")

pytestmark = pytest.mark.gpu

NBH = {"hamming": (ffg.HAMMING, oracle.HAMMING), "adjacent": (ffg.ADJACENT, oracle.ADJACENT)}
F64_L1 = 1e-9      # FP64 rank L1 error bar
F64_CP = 1e-9      # FP64 C_p: |dC_p| <= 2 ||dx||_1 / S_L, well inside this
F32_CP = 1e-5      # FP32 C_p bar


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ffg.build()
    ffg.load()


def _np(t, n=None):
    a = t.cpu().numpy()
    return a if n is None else a[:n]


def run_build(spec, f, nbh):
    sp = ffg.Space.from_spec(spec)
    fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    return ffg.build_graph(sp, fd, NBH[nbh][0]), fd


def assert_same_graph(g, og):
    assert (g.n_raw, g.n_nodes, g.n_edges) == (og.n_raw, og.n_nodes, og.n_edges)
    E = og.n_edges
    np.testing.assert_array_equal(_np(g.node_raw), og.node_raw)
    np.testing.assert_array_equal(_np(g.out_ptr), og.out_ptr)
    np.testing.assert_array_equal(_np(g.in_ptr), og.in_ptr)
    np.testing.assert_array_equal(_np(g.out_idx, E), og.out_idx)
    np.testing.assert_array_equal(_np(g.in_idx, E), og.in_idx)
    np.testing.assert_array_equal(_np(g.outdeg), og.outdeg)
    np.testing.assert_array_equal(_np(g.is_min).astype(bool), og.is_min)
    assert g.n_minima == int(og.is_min.sum())
    assert g.f_opt == og.f_opt


@pytest.mark.parametrize("nbh", ["hamming", "adjacent"])
def test_tiny_spaces_bit_exact(nbh):
    for k, spec in enumerate(fi.tiny_spaces(16, seed0=11000, max_raw=5000)):
        f = fi.runtimes(spec, seed=k + 1, fail_frac=(0.03, 0.3, 0.7)[k % 3],
                        quantum=0.25 if k % 4 == 0 else None)
        og = oracle.build(spec, f, NBH[nbh][1])
        g, _ = run_build(spec, f, nbh)
        assert_same_graph(g, og)


@pytest.mark.parametrize("nbh", ["hamming", "adjacent"])
def test_paper_shaped_spaces(nbh):
    for name, (make, _) in fi.PAPER_SPACES.items():
        spec = make()
        f = fi.runtimes(spec, seed=5, fail_frac=0.7 if name in ("convolution", "gemm") else 0.05)
        og = oracle.build(spec, f, NBH[nbh][1])
        g, fd = run_build(spec, f, nbh)
        assert_same_graph(g, og)
        x, it, res, conv = ffg.pagerank(g, 0.85, 1e-12, prec=ffg.F64)
        assert conv
        xe = oracle.pagerank_exact(og, 0.85)
        assert np.abs(_np(x) - xe).sum() <= F64_L1


@pytest.mark.parametrize("nbh", ["hamming", "adjacent"])
@pytest.mark.parametrize("alpha", [0.5, 0.85, 0.95])
def test_single_small_full_path(nbh, alpha):
    spec = fi.single_small()
    p = [0.0, 0.01, 0.05, 0.1, 0.2]
    for seed in (1, 2, 3):
        f = fi.runtimes(spec, seed)
        og = oracle.build(spec, f, NBH[nbh][1])
        g, fd = run_build(spec, f, nbh)
        assert_same_graph(g, og)
        xe = oracle.pagerank_exact(og, alpha)
        cpe = oracle.centrality(og, xe, p)
        x64, it, res, conv = ffg.pagerank(g, alpha, 1e-12, prec=ffg.F64)
        assert conv and res < 1e-12
        assert np.abs(_np(x64) - xe).sum() <= F64_L1
        assert np.abs(ffg.centrality(g, fd, x64, p) - cpe).max() <= F64_CP
        x32, it32, res32, conv32 = ffg.pagerank(g, alpha, 1e-12, prec=ffg.F32)
        assert conv32 and x32.dtype == torch.float32
        assert np.abs(ffg.centrality(g, fd, x32, p) - cpe).max() <= F32_CP
        assert np.abs(_np(x32).astype(np.float64) - xe).sum() < 1e-4


@pytest.mark.parametrize("nbh", ["hamming", "adjacent"])
def test_single_large_full_size(nbh):
    """2,162,688 raw / 1,419,392 valid points at full size: bit-exact FFG,
    FP64 and FP32 ranks and C_p against the oracle."""
    spec = fi.single_large()
    f = fi.runtimes(spec, 1)
    p = [0.01, 0.05, 0.1]
    og = oracle.build(spec, f, NBH[nbh][1])
    g, fd = run_build(spec, f, nbh)
    assert g.n_nodes == 1419392
    assert_same_graph(g, og)
    xe = oracle.pagerank_exact(og, 0.85)
    cpe = oracle.centrality(og, xe, p)
    x64, it, res, conv = ffg.pagerank(g, 0.85, 1e-12, prec=ffg.F64)
    assert conv
    l1_64 = np.abs(_np(x64) - xe).sum()
    assert l1_64 <= F64_L1
    assert np.abs(ffg.centrality(g, fd, x64, p) - cpe).max() <= F64_CP
    x32, it32, res32, conv32 = ffg.pagerank(g, 0.85, 1e-12, prec=ffg.F32)
    l1_32 = np.abs(_np(x32).astype(np.float64) - xe).sum()
    cp_err = np.abs(ffg.centrality(g, fd, x32, p) - cpe).max()
    print(f"\n{nbh}: FP64 iters {it} L1 {l1_64:.3e}; FP32 iters {it32} L1 {l1_32:.3e} "
          f"C_p err {cp_err:.3e}")
    assert cp_err <= F32_CP


def test_load_balance_groups():
    """Spaces whose mean degree selects each lanes-per-row variant (2/4/8/16)."""
    from ffg_inputs import SpaceSpec
    cases = [
        SpaceSpec("deg2", ("a", "b"), ((1, 2, 3), (1, 2, 3, 4))),                   # mean < 6
        SpaceSpec("deg8", ("a", "b", "c"), (tuple(range(5)), tuple(range(6)), tuple(range(7)))),
        SpaceSpec("deg21", ("a", "b", "c"), (tuple(range(31)), tuple(range(11)), (0, 1, 2, 3))),
        SpaceSpec("deg54", ("a", "b"), (tuple(range(100)), tuple(range(10)))),
    ]
    for spec in cases:
        f = fi.runtimes(spec, 9, fail_frac=0.0, noise_sd=0.3)
        og = oracle.build(spec, f, oracle.HAMMING)
        g, fd = run_build(spec, f, "hamming")
        assert_same_graph(g, og)
        xe = oracle.pagerank_exact(og, 0.85)
        x, it, res, conv = ffg.pagerank(g, 0.85, 1e-13, prec=ffg.F64)
        assert conv and np.abs(_np(x) - xe).sum() <= F64_L1, spec.name


def test_chain_closed_form_on_gpu():
    n, a = 40, 0.85
    spec = fi.SpaceSpec("chain", ("p",), (tuple(range(n)),))
    g, fd = run_build(spec, np.arange(n, 0, -1, dtype=np.float64), "adjacent")
    y = np.array([(1 - a ** (k + 1)) / (1 - a) for k in range(n)])
    x, it, res, conv = ffg.pagerank(g, a, 1e-14, prec=ffg.F64)
    assert np.abs(_np(x) - y / y.sum()).max() < 1e-14
    assert list(ffg.centrality(g, fd, x, [0.0, 1.0])) == [1.0, 1.0]


def test_edge_cases():
    from ffg_inputs import Clause, SpaceSpec
    # no valid configuration
    spec = SpaceSpec("none", ("a",), ((5, 6, 7),), (Clause("prod_le", (0,), (), 1),))
    sp = ffg.Space.from_spec(spec)
    with pytest.raises(ffg.FFGError) as e:
        ffg.build_graph(sp, torch.ones(3, dtype=torch.float64, device="cuda"))
    assert e.value.status == ffg.FFG_ERR_EMPTY
    # one point: a single node without edges, rank 1, C_p 1
    spec = SpaceSpec("one", ("a",), ((3,),))
    g, fd = run_build(spec, np.array([2.0]), "hamming")
    assert (g.n_nodes, g.n_edges, g.n_minima, g.f_opt) == (1, 0, 1, 2.0)
    x, it, res, conv = ffg.pagerank(g, 0.85, 1e-12, prec=ffg.F64)
    assert _np(x)[0] == 1.0 and conv
    assert ffg.centrality(g, fd, x, [0.0])[0] == 1.0
    # everything failed (NaN and 1e10): no edges, no minimum, uniform ranks
    spec = SpaceSpec("fail", ("a", "b"), ((1, 2, 3), (1, 2)))
    f = np.array([1e10, np.nan, 1e10, 2e10, np.nan, 1e10])
    og = oracle.build(spec, f, oracle.HAMMING)
    g, fd = run_build(spec, f, "hamming")
    assert_same_graph(g, og)
    assert g.n_minima == 0 and g.f_opt == np.inf
    x, it, res, conv = ffg.pagerank(g, 0.85, 1e-12, prec=ffg.F64)
    assert np.allclose(_np(x), 1.0 / 6, rtol=0, atol=1e-16)
    with pytest.raises(ffg.FFGError) as e:
        ffg.centrality(g, fd, x, [0.1])
    assert e.value.status == ffg.FFG_ERR_EMPTY
    # 16 parameters (the maximum), negative values, every clause kind
    vals = tuple((-2, 1, 3) if i % 3 == 0 else (1, 2) for i in range(16))
    spec = SpaceSpec("p16", tuple(f"p{i}" for i in range(16)), vals,
                     (Clause("prod_le", (0, 3, 6), (), 4), Clause("prod_ge", (1, 2), (), 2),
                      Clause("divides", (4, 5), (7,)), Clause("prod_le_prod", (9,), (12, 15))))
    for nbh in ("hamming", "adjacent"):
        f = fi.runtimes(spec, 3, fail_frac=0.1)
        og = oracle.build(spec, f, NBH[nbh][1])
        g, fd = run_build(spec, f, nbh)
        assert_same_graph(g, og)
    # products close to the int64 limit
    spec = SpaceSpec("big", ("a", "b", "c"), ((1, 1 << 20, 1 << 31), (1, 3, 1 << 31), (0, 1)),
                     (Clause("prod_le", (0, 1), (), 1 << 40), Clause("divides", (0,), (1,))))
    f = fi.runtimes(spec, 2, fail_frac=0.0)
    og = oracle.build(spec, f, oracle.HAMMING)
    g, fd = run_build(spec, f, "hamming")
    assert_same_graph(g, og)


def test_not_converged_and_warm_start():
    spec = fi.single_small()
    f = fi.runtimes(spec, 4)
    og = oracle.build(spec, f, oracle.HAMMING)
    g, fd = run_build(spec, f, "hamming")
    # three iterations only: status NOT_CONVERGED, ranks = three power steps
    x, it, res, conv = ffg.pagerank(g, 0.85, 1e-12, max_iter=3, prec=ffg.F64)
    assert not conv and it == 3
    xo, ito, reso, convo = oracle.pagerank_power(og, 0.85, 1e-12, max_iter=3)
    assert ito == 3 and abs(res - reso) < 1e-14
    assert np.abs(_np(x) - xo / xo.sum()).sum() < 1e-14
    # warm start from the exact solution: converges at once
    xe = oracle.pagerank_exact(og, 0.85)
    x, it, res, conv = ffg.pagerank(g, 0.85, 1e-12, prec=ffg.F64,
                                    init=torch.from_numpy(xe).cuda())
    assert conv and it <= 2 and np.abs(_np(x) - xe).sum() <= F64_L1


def test_deterministic():
    spec = fi.single_large()
    f = fi.runtimes(spec, 2)
    g, fd = run_build(spec, f, "hamming")
    a = ffg.pagerank(g, 0.85, 1e-12, prec=ffg.F32)[0].clone()
    b = ffg.pagerank(g, 0.85, 1e-12, prec=ffg.F32)[0]
    assert torch.equal(a, b)
    g2, _ = run_build(spec, f, "hamming")
    assert torch.equal(g.in_idx, g2.in_idx) and torch.equal(g.out_idx, g2.out_idx)


def test_async_solve_and_query():
    spec = fi.single_small()
    f = fi.runtimes(spec, 6)
    g, fd = run_build(spec, f, "hamming")
    need = ffg.pagerank_workspace_bytes(g.n_nodes, g.n_edges, ffg.F64)
    ws = ffg.workspace(need)
    x = torch.empty(g.n_nodes, dtype=torch.float64, device="cuda")
    st, it, res = ffg.pagerank_solve(g.c, 0.85, 1e-12, 1000, ffg.F64, x.data_ptr(), 0,
                                     ws.data_ptr(), need, sync=False,
                                     stream=torch.cuda.current_stream().cuda_stream)
    assert st == 0 and it is None
    st, it, res = ffg.pagerank_query(ws.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 0 and it > 10 and res < 1e-12


def test_centrality_many_thresholds():
    """The largest threshold list (32 values, unsorted, with repeats)."""
    spec = fi.single_small()
    f = fi.runtimes(spec, 8, fail_frac=0.1)
    og = oracle.build(spec, f, oracle.HAMMING)
    g, fd = run_build(spec, f, "hamming")
    p = list(np.linspace(0.3, 0.0, 30)) + [0.05, 0.05]
    xe = oracle.pagerank_exact(og, 0.85)
    x, *_ = ffg.pagerank(g, 0.85, 1e-12, prec=ffg.F64)
    assert np.abs(ffg.centrality(g, fd, x, p) - oracle.centrality(og, xe, p)).max() <= F64_CP


def test_prepared_layout_and_damping_sweep():
    """One pagerank_prepare, then solves at several damping factors reuse it."""
    spec = fi.single_small()
    f = fi.runtimes(spec, 10, fail_frac=0.2)
    og = oracle.build(spec, f, oracle.HAMMING)
    g, fd = run_build(spec, f, "hamming")
    need = ffg.pagerank_workspace_bytes(g.n_nodes, g.n_edges, ffg.F64)
    ws = ffg.workspace(need)
    assert ffg.pagerank_prepare(g.c, ffg.F64, ws.data_ptr(), need,
                                torch.cuda.current_stream().cuda_stream) == 0
    for alpha in (0.5, 0.7, 0.85, 0.95):
        x, it, res, conv = ffg.pagerank(g, alpha, 1e-13, prec=ffg.F64, ws=ws, prepared=True)
        assert conv and np.abs(_np(x) - oracle.pagerank_exact(og, alpha)).sum() <= F64_L1


def test_batched_pagerank_matches_oracle():
    """Many jobs of uneven size, shared graphs, several dampings, one launch."""
    specs, refs = [], []
    cases = [(fi.single_small(), 1), (fi.pnpoly_space(), 2), (fi.conv_mi50_space(), 3),
             (fi.gemm_space(), 4)] + [(sp, 10 + k) for k, sp in
                                      enumerate(fi.tiny_spaces(6, seed0=13000, max_raw=3000))]
    graphs = []
    for spec, seed in cases:
        f = fi.runtimes(spec, seed, fail_frac=0.7 if spec.name == "gemm" else 0.05)
        for nbh in ("hamming", "adjacent"):
            og = oracle.build(spec, f, NBH[nbh][1])
            g, fd = run_build(spec, f, nbh)
            graphs.append((g, og))
    for k, (g, og) in enumerate(graphs):
        for alpha in ((0.5, 0.85) if k % 2 else (0.95,)):
            specs.append((g, alpha))
            refs.append(oracle.pagerank_exact(og, alpha))
    for prec, bar in ((ffg.F64, F64_L1), (ffg.F32, 1e-5)):
        batch = ffg.PageRankBatch(specs, prec=prec, tol=1e-12)
        for _ in range(2):          # a plan can be run again
            batch.run()
            it, res, st = batch.query()
            assert (st == ffg.FFG_OK).all(), st
            for x, xe in zip(batch.ranks, refs):
                assert np.abs(_np(x).astype(np.float64) - xe).sum() <= bar


def test_batched_pagerank_large_jobs_share_blocks():
    """A large job (several dedicated blocks) next to small ones."""
    spec = fi.single_large()
    f = fi.runtimes(spec, 1)
    og = oracle.build(spec, f, oracle.ADJACENT)
    g, fd = run_build(spec, f, "adjacent")
    small = fi.single_small()
    fs = fi.runtimes(small, 2)
    ogs = oracle.build(small, fs, oracle.HAMMING)
    gs, _ = run_build(small, fs, "hamming")
    batch = ffg.PageRankBatch([(g, 0.85), (gs, 0.85), (gs, 0.6)], prec=ffg.F64, tol=1e-12)
    assert batch.plan.n_blocks > 3
    batch.run()
    it, res, st = batch.query()
    assert (st == 0).all()
    assert np.abs(_np(batch.ranks[0]) - oracle.pagerank_exact(og, 0.85)).sum() <= F64_L1
    assert np.abs(_np(batch.ranks[1]) - oracle.pagerank_exact(ogs, 0.85)).sum() <= F64_L1
    assert np.abs(_np(batch.ranks[2]) - oracle.pagerank_exact(ogs, 0.6)).sum() <= F64_L1


def test_batched_centrality_matches_single():
    p = [0.0, 0.01, 0.05, 0.2, 0.1]
    specs, refs = [], []
    for k, spec in enumerate([fi.single_small(), fi.pnpoly_space(), fi.conv_mi50_space()]):
        f = fi.runtimes(spec, k + 3)
        og = oracle.build(spec, f, oracle.HAMMING)
        g, fd = run_build(spec, f, "hamming")
        x, *_ = ffg.pagerank(g, 0.85, 1e-12, prec=ffg.F64)
        specs.append((g, fd, x))
        refs.append(oracle.centrality(og, oracle.pagerank_exact(og, 0.85), p))
    out = ffg.centrality_many(specs, p)
    for row, ref in zip(out, refs):
        assert np.abs(row - ref).max() <= F64_CP


def test_bounded_wait_reports_timeout():
    """Fault injected on the host: the plan is edited so that one block of a
    multi-block job never starts.  The job's other block gives up at the
    bounded barrier and the host reads FFG_ERR_TIMEOUT; the context stays
    usable."""
    spec = fi.single_large()
    g, _ = run_build(spec, fi.runtimes(spec, 1), "adjacent")
    small = fi.single_small()
    gs, _ = run_build(small, fi.runtimes(small, 2), "hamming")
    batch = ffg.PageRankBatch([(g, 0.85), (gs, 0.85)], prec=ffg.F32)
    batch.replan((1.0, 1.0, 0, 8, 1))   # claim order
    ws_base = batch.ws.data_ptr()
    items = batch.ws[batch.plan.items - ws_base:].view(torch.int32)
    # the large job's ranks are claimed first: (0, 0), (0, 1), ...
    assert items[0].item() == 0 and items[1].item() == 0
    assert items[2].item() == 0 and items[3].item() == 1
    batch.plan.n_items = 1        # only rank 0 of the large job is ever claimed
    torch.cuda.synchronize()
    batch.run()
    st, it, res, sts = ffg.pagerank_batch_query(batch.plan,
                                                torch.cuda.current_stream().cuda_stream)
    assert st == ffg.FFG_ERR_TIMEOUT and sts[0] == ffg.FFG_ERR_TIMEOUT
    # the device is still usable: a fresh plan runs to convergence
    fresh = ffg.PageRankBatch([(g, 0.85), (gs, 0.85)], prec=ffg.F32)
    fresh.run()
    it, res, sts = fresh.query()
    assert (sts == ffg.FFG_OK).all()


def test_group_waits_for_a_long_earlier_job():
    """A group's blocks wait for a rank that is busy with an earlier job for as
    long as that job runs: a bounded wait gives up only when no block makes
    progress.  Job A (PnPoly, 8184 nodes, FP64, tol 0: it runs all of
    max_iter, several seconds, on one block) is claimed first; job B (1.42M
    nodes) has a rank on every block, one of them A's, so B's other ranks wait
    at B's first barrier longer than the 2 s a wait without progress may last.
    Both finish, and B gives the bits of a solve of B alone."""
    small, big = fi.pnpoly_space(), fi.single_large()
    ga, _ = run_build(small, fi.runtimes(small, 3), "hamming")
    gb, _ = run_build(big, fi.runtimes(big, 1), "adjacent")
    batch = ffg.PageRankBatch([(ga, 0.85), (gb, 0.85)], prec=ffg.F64, tol=1e-12)
    batch.jobs[0].tol = 0.0
    batch.jobs[0].max_iter = 60000
    # min_tiles 12 keeps A on one block and still spreads B over every block
    batch.replan((0.01, 0.001, 0, 24, 1, 0, 12), job_cost=[100.0, 10.0])
    assert batch.plan.n_items == 1 + batch.plan.n_blocks   # A alone, B on every block
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    batch.run()
    e1.record()
    e1.synchronize()
    st, it, res, sts = ffg.pagerank_batch_query(batch.plan,
                                                torch.cuda.current_stream().cuda_stream)
    ms = e0.elapsed_time(e1)
    print(f"\nA {it[0]} iterations, B {it[1]} iterations, {ms:.0f} ms")
    assert sts[0] == ffg.FFG_ERR_NOT_CONVERGED and it[0] == 60000
    assert sts[1] == ffg.FFG_OK
    assert ms > 2100.0, ms   # B's ranks did wait longer than the limit
    ref = ffg.PageRankBatch([(gb, 0.85)], prec=ffg.F64, tol=1e-12)
    ref.run()
    it_r, _, st_r = ref.query()
    assert st_r[0] == ffg.FFG_OK and it_r[0] == it[1]
    np.testing.assert_array_equal(_np(batch.ranks[1]), _np(ref.ranks[0]))


def test_precision_form_at_scale():
    """11 parameters, 19.5M raw / 12.8M valid points, Hamming: the FFG is
    bit-exact; FP32 ranks (FP64/exact reductions) and C_p are compared with the
    oracle's exact FP64 solve, and so are the FP64 ranks."""
    spec = fi.precision_large()
    f = fi.runtimes(spec, 1)
    p = [0.01, 0.05, 0.10]
    og = oracle.build(spec, f, oracle.HAMMING)
    g, fd = run_build(spec, f, "hamming")
    assert g.n_nodes == 12774528
    assert_same_graph(g, og)
    xe = oracle.pagerank_exact(og, 0.85)
    cpe = oracle.centrality(og, xe, p)
    x32, it32, res32, conv32 = ffg.pagerank(g, 0.85, 1e-12, prec=ffg.F32)
    l1_32 = float(np.abs(_np(x32).astype(np.float64) - xe).sum())
    cp32 = ffg.centrality(g, fd, x32, p)
    x64, it64, res64, conv64 = ffg.pagerank(g, 0.85, 1e-12, prec=ffg.F64)
    l1_64 = float(np.abs(_np(x64) - xe).sum())
    print(f"\nprecision form: N={g.n_nodes} E={g.n_edges}; FP32 iters {it32} rank L1 {l1_32:.3e} "
          f"C_p err {np.abs(cp32 - cpe).max():.3e}; FP64 iters {it64} rank L1 {l1_64:.3e}")
    assert conv32 and conv64
    assert np.abs(cp32 - cpe).max() <= F32_CP
    assert l1_64 <= F64_L1


def test_batch_tuning_changes_schedule_not_results():
    specs, refs = [], []
    for k, spec in enumerate([fi.single_small(), fi.pnpoly_space(), fi.conv_mi50_space()]):
        f = fi.runtimes(spec, 20 + k)
        og = oracle.build(spec, f, oracle.HAMMING)
        g, _ = run_build(spec, f, "hamming")
        for alpha in (0.7, 0.9):
            specs.append((g, alpha))
            refs.append(oracle.pagerank_exact(og, alpha))
    batch = ffg.PageRankBatch(specs, prec=ffg.F64, tol=1e-12)
    first = {}
    for tuning in ((1.0, 1.0, 0), (0.1, 0.1, 0), (5.0, 1.0, 3), (1.0, 1.0, 0, 8),
                   (0.1, 0.1, 0, 8), (0.1, 0.1, 0, 8, 1), (0.5, 0.5, 0, 24, 1),
                   (1.0, 1.0, 0, 16), (0.1, 0.02, 0, 16, 0), (0.5, 0.5, 0, 16, 1),
                   (1.0, 1.0, 0, 8, 0, 2), (0.1, 0.02, 0, 24, 0, 2), (0.1, 0.02, 0, 16, 0, 2),
                   (1.0, 1.0, 0, 24, 2), (1.0, 1.0, 0, 16, 2), (1.0, 1.0, 0, 24, 2, 2),
                   (0.05, 0.005, 0, 24, 1, 0, 4), (0.02, 0.002, 0, 16, 0, 0, 8),
                   (0.01, 0.001, 0, 8, 1, 2, 2)):
        batch.replan(tuning)
        batch.run()
        it, res, st = batch.query()
        assert (st == 0).all()
        xs = [_np(x) for x in batch.ranks]
        for x, xe in zip(xs, refs):
            assert np.abs(x - xe).sum() <= F64_L1
        # fixed-point reductions and exact FP64 in-sums: the schedule does not
        # change a single bit (the storage form of w may change the last one)
        form = tuning[5] if len(tuning) > 5 else 0
        if form not in first:
            first[form] = (it.copy(), xs)
        else:
            np.testing.assert_array_equal(it, first[form][0])
            for x, x0 in zip(xs, first[form][1]):
                np.testing.assert_array_equal(x, x0)


def test_batch_sweep_order_fp32_bit_exact():
    """The sweep order (every job one step per phase on the whole grid, units
    taken across blocks) gives the FP32 bits of the per-block lists, on jobs
    of very different sizes and dampings, and repeats them run after run."""
    specs, refs = [], []
    cases = [(fi.single_large(), 1, "adjacent"), (fi.gemm_space(), 2, "hamming"),
             (fi.single_small(), 3, "hamming"), (fi.pnpoly_space(), 4, "adjacent")]
    for spec, seed, nbh in cases:
        f = fi.runtimes(spec, seed, fail_frac=0.7 if spec.name == "gemm" else 0.03)
        og = oracle.build(spec, f, NBH[nbh][1])
        g, _ = run_build(spec, f, nbh)
        for alpha in (0.5, 0.85, 0.95):
            specs.append((g, alpha))
            refs.append((og, alpha))
    batch = ffg.PageRankBatch(specs, prec=ffg.F32, tol=1e-12)
    out = {}
    for tuning in ((0.05, 0.005, 0, 24, 0), (1.0, 1.0, 0, 24, 2), (1.0, 1.0, 0, 16, 2)):
        batch.replan(tuning)
        for _ in range(2):
            batch.run()
            it, res, st = batch.query()
            assert (st == 0).all()
            xs = [_np(x) for x in batch.ranks]
            if "ref" not in out:
                out["ref"] = (it.copy(), res.copy(), xs)
            np.testing.assert_array_equal(it, out["ref"][0])
            np.testing.assert_array_equal(res, out["ref"][1])
            for x, x0 in zip(xs, out["ref"][2]):
                np.testing.assert_array_equal(x, x0)
    for x, (og, alpha) in zip(out["ref"][2], refs):
        assert np.abs(x.astype(np.float64) - oracle.pagerank_exact(og, alpha)).sum() <= 1e-5


def test_batch_measured_costs_change_schedule_not_results():
    """The per-job block-seconds of a run, fed back as job costs, give
    another schedule and the same bits (FP32 and FP64); no block is busy
    with two jobs at once, so the busy times add up to at most the grid's
    time."""
    specs = []
    for k, spec in enumerate([fi.single_small(), fi.pnpoly_space(), fi.conv_mi50_space(),
                              fi.gemm_space()]):
        f = fi.runtimes(spec, 30 + k, fail_frac=0.7 if spec.name == "gemm" else 0.05)
        g, _ = run_build(spec, f, "hamming" if k % 2 == 0 else "adjacent")
        for alpha in (0.6, 0.85):
            specs.append((g, alpha))
    for prec in (ffg.F32, ffg.F64):
        batch = ffg.PageRankBatch(specs, prec=prec, tol=1e-12)
        batch.replan((0.1, 0.1, 0, 16))
        batch.run()
        batch.query()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        batch.run()
        e1.record()
        it0, _, st = batch.query()
        assert (st == 0).all()
        xs0 = [_np(x) for x in batch.ranks]
        busy = batch.times()
        assert busy.shape == (len(specs),) and (busy > 0).all()
        wall = e0.elapsed_time(e1) / 1e3
        assert busy.sum() <= batch.plan.n_blocks * wall * 1.01 + 1e-4
        n_blocks0 = batch.plan.n_blocks
        for cost in (busy, busy[::-1].copy(), np.linspace(1.0, 50.0, len(specs))):
            batch.replan((0.1, 0.1, 0, 16), job_cost=cost)
            batch.run()
            it, _, st = batch.query()
            assert (st == 0).all()
            np.testing.assert_array_equal(it, it0)
            for x, x0 in zip(batch.ranks, xs0):
                np.testing.assert_array_equal(_np(x), x0)
        assert batch.plan.n_blocks == n_blocks0


def test_batch_job_table_forms_agree():
    """A batch of up to FFG_PR_PARAM_JOBS jobs passes its job table to the
    kernel as parameters, a larger one reads it from device memory: the same
    jobs give the same bits either way, in every block width and order."""
    cases = [(fi.single_small(), 5, "hamming"), (fi.pnpoly_space(), 6, "adjacent"),
             (fi.conv_mi50_space(), 7, "hamming")]
    graphs, refs = [], []
    for spec, seed, nbh in cases:
        f = fi.runtimes(spec, seed)
        og = oracle.build(spec, f, NBH[nbh][1])
        g, _ = run_build(spec, f, nbh)
        graphs.append(g)
        refs.append(og)
    dampings = np.linspace(0.5, 0.95, 81)
    jobs = [(g, float(a)) for g in graphs for a in dampings]
    assert len(jobs) > ffg.PARAM_JOBS
    big = ffg.PageRankBatch(jobs, prec=ffg.F32, tol=1e-12)
    small = ffg.PageRankBatch(jobs[:ffg.PARAM_JOBS], prec=ffg.F32, tol=1e-12)
    assert big.plan.param_jobs == 0 and small.plan.param_jobs == ffg.PARAM_JOBS
    for tuning in ((1.0, 1.0, 0, 8, 0), (0.1, 0.02, 0, 24, 0), (0.5, 0.5, 0, 16, 1),
                   (1.0, 1.0, 0, 24, 2), (1.0, 1.0, 0, 16, 2)):
        out = []
        for b in (big, small):
            b.replan(tuning)
            b.run()
            it, _, st = b.query()
            assert (st == 0).all()
            out.append((it, [_np(x) for x in b.ranks]))
        np.testing.assert_array_equal(out[0][0][:ffg.PARAM_JOBS], out[1][0])
        for x0, x1 in zip(out[0][1], out[1][1]):
            np.testing.assert_array_equal(x0, x1)
    for k in (0, 80, 81 + 40, 2 * 81 + 80):    # against the exact solve
        xe = oracle.pagerank_exact(refs[k // 81], float(dampings[k % 81]))
        assert np.abs(_np(big.ranks[k]).astype(np.float64) - xe).sum() <= 1e-5


def test_batch_run_one_call_matches_separate_calls():
    """ffg_batch_run -- every FFG, every solve, every C_p in one call -- is
    bit-exact against the oracle's graphs, within the FP64 bars of its
    ranks and C_p, and gives the bits of the separate calls; its
    launches-only form replays from a CUDA graph."""
    cases = [(fi.single_small(), 1, 0.03), (fi.pnpoly_space(), 2, 0.7),
             (fi.conv_mi50_space(), 3, 0.3)]
    cases += [(sp, 40 + k, 0.03) for k, sp in
              enumerate(fi.tiny_spaces(5, seed0=15000, max_raw=3000))]
    p = [0.0, 0.01, 0.05, 0.1]
    specs, refs = [], []
    for k, (spec, seed, fail) in enumerate(cases):
        f = fi.runtimes(spec, seed, fail_frac=fail)
        nbh = "hamming" if k % 2 == 0 else "adjacent"
        try:
            og = oracle.build(spec, f, NBH[nbh][1])
        except oracle.OracleError:      # a space without valid configurations
            continue
        if not og.is_min.any():
            continue
        fd = torch.from_numpy(f).cuda()
        specs.append((ffg.Space.from_spec(spec), fd, NBH[nbh][0]))
        xe = oracle.pagerank_exact(og, 0.85)
        refs.append((og, xe, oracle.centrality(og, xe, p)))
    bb = ffg.BuildBatch(specs)
    batch = ffg.PageRankBatch([(g, 0.85) for g in bb.graphs], prec=ffg.F64, tol=1e-12)
    cp_specs = [(g, fd, x) for g, (_, fd, _), x in zip(bb.graphs, specs, batch.ranks)]
    cpb = ffg.CentralityBatch(cp_specs, p)
    sb = ffg.SpaceBatch(batch, builds=bb, cp=cpb)
    for g in bb.graphs:
        g.out_idx.fill_(-1)
        g.in_ptr.fill_(-1)
    st, out = sb.run()
    assert st == ffg.FFG_OK, ffg.ffg_last_error()
    assert (out["build_status"] == 0).all() and (out["pr_status"] == 0).all()
    for g, x, (og, xe, cpe) in zip(bb.graphs, batch.ranks, refs):
        assert_same_graph(g, og)
        assert np.abs(_np(x) - xe).sum() <= F64_L1
    for row, (_, _, cpe) in zip(out["cp"], refs):
        assert np.abs(row - cpe).max() <= F64_CP
    xs = [_np(x) for x in batch.ranks]
    # the separate calls: the same bits
    bb.rerun()
    batch.run()
    it, res, sts = batch.query()
    np.testing.assert_array_equal(it, out["iters"])
    np.testing.assert_array_equal(res, out["residual"])
    for x, x0 in zip(batch.ranks, xs):
        np.testing.assert_array_equal(_np(x), x0)
    np.testing.assert_array_equal(ffg.centrality_many(cp_specs, p), out["cp"])
    # launches only -- builds, solves and C_p -- captured and replayed
    cg = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(cg, stream=side):
            sb.run(sync=False, stream=side)
    torch.cuda.current_stream().wait_stream(side)
    for g, x in zip(bb.graphs, batch.ranks):
        g.in_idx.fill_(-1)
        x.fill_(0)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(cpb.query()[0], out["cp"])
    # the plan's device results are overwritten (NaN bytes) before the replay
    off = cpb.plan.cp - cpb.ws.data_ptr()
    cpb.ws[off:off + 8 * cpb.plan.n_jobs * cpb.plan.n_p].fill_(0xff)
    assert np.isnan(cpb.query()[0]).all()
    cg.replay()
    torch.cuda.synchronize()
    for g, x, x0, (og, _, _) in zip(bb.graphs, batch.ranks, xs, refs):
        assert_same_graph(g, og)
        np.testing.assert_array_equal(_np(x), x0)
    cp_replay, sts = cpb.query()
    assert (sts == 0).all()
    np.testing.assert_array_equal(cp_replay, out["cp"])
    for row, (_, _, cpe) in zip(cp_replay, refs):
        assert np.abs(row - cpe).max() <= F64_CP


def test_batched_build_matches_per_space_builds():
    """All FFGs of many spaces at once (both neighbourhoods, ragged sizes,
    failures and ties): bit-exact against the oracle; a re-run from the
    workspace, plain and replayed from a CUDA graph, gives the same arrays."""
    cases = [(fi.single_small(), 1, 0.03, None), (fi.pnpoly_space(), 2, 0.7, None),
             (fi.conv_mi50_space(), 3, 0.3, 0.25), (fi.gemm_space(), 4, 0.7, None)]
    cases += [(sp, 10 + k, (0.03, 0.3, 0.7)[k % 3], 0.5 if k % 4 == 0 else None)
              for k, sp in enumerate(fi.tiny_spaces(12, seed0=14000, max_raw=4000))]
    specs, fits, refs = [], [], []
    for k, (spec, seed, fail, quantum) in enumerate(cases):
        f = fi.runtimes(spec, seed, fail_frac=fail, quantum=quantum)
        nbh = "hamming" if k % 2 == 0 else "adjacent"
        og = oracle.build(spec, f, NBH[nbh][1])
        if og.n_nodes == 0:
            continue
        fd = torch.from_numpy(f).cuda()
        fits.append(fd)
        specs.append((ffg.Space.from_spec(spec), fd, NBH[nbh][0]))
        refs.append(og)
    bb = ffg.BuildBatch(specs)
    for g, og in zip(bb.graphs, refs):
        assert_same_graph(g, og)
    # re-run: clobber the arrays first, the re-run must restore them
    for g in bb.graphs:
        g.out_idx.fill_(-1)
        g.in_ptr.fill_(-1)
    bb.rerun()
    st, sts = bb.query()
    assert st == ffg.FFG_OK and (sts == 0).all()
    for g, og in zip(bb.graphs, refs):
        assert_same_graph(g, og)
    cg = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(cg, stream=side):
            bb.rerun(stream=side)
    torch.cuda.current_stream().wait_stream(side)
    for g in bb.graphs:
        g.out_idx.fill_(-1)
    cg.replay()
    torch.cuda.synchronize()
    for g, og in zip(bb.graphs, refs):
        assert_same_graph(g, og)


def test_batched_build_rerun_refuses_changed_sizes():
    """A re-run whose counts no longer match the arrays (fitness changed)
    leaves that graph untouched and reports it; the others are rebuilt."""
    a, b = fi.single_small(), fi.conv_mi50_space()
    fa = torch.from_numpy(fi.runtimes(a, 1)).cuda()
    fb = torch.from_numpy(fi.runtimes(b, 2)).cuda()
    bb = ffg.BuildBatch([(ffg.Space.from_spec(a), fa, ffg.HAMMING),
                         (ffg.Space.from_spec(b), fb, ffg.HAMMING)])
    before = [_np(t).copy() for t in (bb.graphs[0].out_ptr, bb.graphs[0].out_idx)]
    fa.copy_(torch.from_numpy(fi.runtimes(a, 99)))   # other edges, other edge count
    og_b = oracle.build(b, fi.runtimes(b, 2), oracle.HAMMING)
    bb.graphs[1].out_idx.fill_(-1)
    bb.rerun()
    st, sts = bb.query()
    assert st == ffg.FFG_ERR_INVALID_ARG and sts[0] == ffg.FFG_ERR_INVALID_ARG and sts[1] == 0
    np.testing.assert_array_equal(_np(bb.graphs[0].out_ptr), before[0])
    np.testing.assert_array_equal(_np(bb.graphs[0].out_idx), before[1])
    assert_same_graph(bb.graphs[1], og_b)


def _longest_path(og):
    key = np.where(og.failed, np.inf, og.node_fit)
    depth = np.zeros(og.n_nodes, dtype=np.int64)
    for v in np.argsort(-key, kind="stable"):
        a, b = og.in_ptr[v], og.in_ptr[v + 1]
        if b > a:
            depth[v] = 1 + depth[og.in_idx[a:b]].max()
    return int(depth.max())


@pytest.mark.parametrize("nbh", ["hamming", "adjacent"])
def test_dag_solve_bit_exact(nbh):
    """The level-by-level exact solve reproduces the sequential one bit for
    bit (y for d < 1 and d = 1, and the absorbing walk); its PageRank mode is
    the exact PageRank and the power iteration's limit; its level count is
    the longest improving path + 1."""
    cases = [(fi.single_small(), 1, 0.03), (fi.pnpoly_space(), 2, 0.7),
             (fi.gemm_space(), 3, 0.3)]
    cases += [(sp, 20 + k, (0.03, 0.3, 0.7)[k % 3])
              for k, sp in enumerate(fi.tiny_spaces(8, seed0=15000, max_raw=3000))]
    for spec, seed, fail in cases:
        f = fi.runtimes(spec, seed, fail_frac=fail)
        try:
            og = oracle.build(spec, f, NBH[nbh][1])
        except oracle.OracleError:      # a space without valid configurations
            continue
        g, fd = run_build(spec, f, nbh)
        for d in (0.5, 0.85, 1.0):
            y, lv = ffg.dag(g, d, ffg.DAG_VALUES)
            np.testing.assert_array_equal(_np(y), oracle.dag_values(og, d))
        assert lv == _longest_path(og) + 1
        a, _ = ffg.dag(g, 1.0, ffg.DAG_ABSORB)
        ae = oracle.absorption(og)
        np.testing.assert_array_equal(_np(a), ae)
        x, _ = ffg.dag(g, 0.85, ffg.DAG_PAGERANK)
        assert np.abs(_np(x) - oracle.pagerank_exact(og, 0.85)).sum() <= 1e-14
        if og.is_min.any():
            p = [0.0, 0.05, 0.2]
            cp = ffg.centrality(g, fd, a, p)
            assert np.abs(cp - oracle.centrality(og, ae, p)).max() <= 1e-12


def test_dag_solve_full_size():
    """Both neighbourhoods of the single large space: bit-exact y, and the
    exact PageRank agrees with the FP64 power iteration."""
    spec = fi.single_large()
    f = fi.runtimes(spec, 1)
    for nbh in ("hamming", "adjacent"):
        og = oracle.build(spec, f, NBH[nbh][1])
        g, _ = run_build(spec, f, nbh)
        y, lv = ffg.dag(g, 0.85, ffg.DAG_VALUES)
        np.testing.assert_array_equal(_np(y), oracle.dag_values(og, 0.85))
        x, _ = ffg.dag(g, 0.85, ffg.DAG_PAGERANK)
        xp, it, res, conv = ffg.pagerank(g, 0.85, 1e-13, prec=ffg.F64)
        assert conv and np.abs(_np(x) - _np(xp)).sum() <= 1e-11
        a, _ = ffg.dag(g, 1.0, ffg.DAG_ABSORB)
        np.testing.assert_array_equal(_np(a), oracle.absorption(og))


def test_walks_bit_exact_and_unbiased():
    """Simulated improving walks: counts and moves equal the oracle's (same
    SplitMix64 draws) on paper-shaped spaces and the 1.42M-node space; the
    arrival frequencies of 10^7 walks on that space lie within binomial
    bounds of the exact absorbing walk."""
    cases = [(fi.single_small(), 1, "hamming", 100_000), (fi.pnpoly_space(), 2, "adjacent", 100_000),
             (fi.gemm_space(), 3, "hamming", 50_000), (fi.single_large(), 1, "hamming", 1_000_000)]
    for spec, seed, nbh, W in cases:
        f = fi.runtimes(spec, seed)
        og = oracle.build(spec, f, NBH[nbh][1])
        g, _ = run_build(spec, f, nbh)
        counts, steps = ffg.walks(g, seed=77 + seed, n_walks=W)
        ce, se = oracle.walks(og, seed=77 + seed, n_walks=W)
        np.testing.assert_array_equal(_np(counts).astype(np.uint64), ce)
        assert steps == se
    W = 10_000_000
    counts, _ = ffg.walks(g, seed=5, n_walks=W)
    a, _ = ffg.dag(g, 1.0, ffg.DAG_ABSORB)
    a = _np(a)
    sinks = _np(g.outdeg) == 0
    freq = _np(counts)[sinks] / W
    p = a[sinks]
    sd = np.sqrt(np.clip(p * (1 - p), 0.0, None) / W)
    assert (np.abs(freq - p) <= 6 * sd + 1e-12).all()


def test_minima_fraction_bit_exact():
    for spec, seed, nbh in [(fi.single_small(), 1, "hamming"), (fi.gemm_space(), 2, "adjacent"),
                            (fi.single_large(), 1, "hamming")]:
        f = fi.runtimes(spec, seed)
        og = oracle.build(spec, f, NBH[nbh][1])
        g, fd = run_build(spec, f, nbh)
        frac, node = ffg.minima_fraction(g, fd)
        np.testing.assert_array_equal(_np(frac), oracle.minima_fraction(og))
        np.testing.assert_array_equal(_np(node), np.flatnonzero(og.is_min))


def test_graph_checkpoint_resumes_on_gpu(tmp_path):
    """An FFG saved as a CSR .npz and loaded back onto the GPU is the same
    graph and gives the same ranks bit for bit; a solve resumed from saved
    ranks converges at once."""
    spec = fi.pnpoly_space()
    f = fi.runtimes(spec, 9, fail_frac=0.3)
    og = oracle.build(spec, f, oracle.HAMMING)
    g, _ = run_build(spec, f, "hamming")
    x, it, res, conv = ffg.pagerank(g, 0.85, 1e-12, prec=ffg.F64)
    path = tmp_path / "ffg.npz"
    g.save(path)
    np.save(tmp_path / "ranks.npy", _np(x))
    h = ffg.load_graph(path, device="cuda")
    assert_same_graph(h, og)
    y, it2, res2, conv2 = ffg.pagerank(h, 0.85, 1e-12, prec=ffg.F64)
    assert conv and conv2 and it2 == it
    np.testing.assert_array_equal(_np(y), _np(x))
    x0 = torch.from_numpy(np.load(tmp_path / "ranks.npy")).cuda()
    z, it3, res3, conv3 = ffg.pagerank(h, 0.85, 1e-12, prec=ffg.F64, init=x0)
    assert conv3 and it3 <= 2
    assert np.abs(_np(z) - oracle.pagerank_exact(og, 0.85)).sum() <= F64_L1


def test_row_partitioned_fp64_equals_single_solve():
    """The row-partitioned form (several ranges, one process standing for
    several ranks) gives pagerank_solve's FP64 ranks bit for bit: the same
    exact fixed-point sums, the same stopping decisions."""
    from paper_2210_01465_gb300.multi import solve_rows, split_rows
    cases = [(fi.single_small(), 2, "hamming", 3), (fi.pnpoly_space(), 3, "adjacent", 5),
             (fi.single_large(), 1, "hamming", 4)]
    for spec, seed, nbh, parts in cases:
        f = fi.runtimes(spec, seed, fail_frac=0.3 if parts == 5 else 0.03)
        g, _ = run_build(spec, f, nbh)
        x, it, res, conv = ffg.pagerank(g, 0.85, 1e-12, prec=ffg.F64)
        bounds = split_rows(_np(g.in_ptr), parts)
        for ranges in (bounds, [(0, g.n_nodes)]):
            y, it2, res2, conv2 = solve_rows(g, ranges, 0.85, 1e-12, prec=ffg.F64)
            assert conv2 and it2 == it and res2 == res
            np.testing.assert_array_equal(_np(y), _np(x))


def test_row_partitioned_fp32_and_warm_start():
    """FP32 over ranges (tile groupings differ from the single solve, so the
    FP32 sums are not bit-identical): C_p within the FP32 bar of the oracle's
    exact solve; a warm start from the exact ranks converges at once; tiny
    ranges (one row, rows without in-edges) work."""
    from paper_2210_01465_gb300.multi import solve_rows, split_rows
    spec = fi.conv_mi50_space()
    f = fi.runtimes(spec, 11)
    og = oracle.build(spec, f, oracle.HAMMING)
    g, fd = run_build(spec, f, "hamming")
    xe = oracle.pagerank_exact(og, 0.85)
    p = [0.0, 0.05, 0.1]
    cpe = oracle.centrality(og, xe, p)
    n = g.n_nodes
    for ranges in (split_rows(_np(g.in_ptr), 4), [(0, 1), (1, 2), (2, n)]):
        y, it, res, conv = solve_rows(g, ranges, 0.85, 1e-12, prec=ffg.F32)
        assert conv
        assert np.abs(_np(y).astype(np.float64) - xe).sum() < 1e-5
        cp = ffg.centrality(g, fd, y, p)
        assert np.abs(cp - cpe).max() <= F32_CP
    y, it, res, conv = solve_rows(g, split_rows(_np(g.in_ptr), 3), 0.85, 1e-12, prec=ffg.F64,
                                  init=torch.from_numpy(xe).cuda())
    assert conv and it <= 2 and np.abs(_np(y) - xe).sum() <= F64_L1
