"""PageRank through the entry point that allocates nothing.

pagerank_solve_static serves callers that cannot allocate device memory
(another component owns the device memory, or cudaMalloc is not allowed or
would synchronise the device where they run).  Its scratch space is a
fixed device array inside the library.  This file is collected last so that
a run stopping at the first failure has already run every other test; it
also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import ffg_inputs as fi

torch = pytest.importorskip("torch")
ffg = pytest.importorskip("paper_2210_01465_gb300")

pytestmark = pytest.mark.gpu

F64_L1 = 1e-9     # the FP64 rank bar used by the parity tests
F32_L1 = 1e-6     # the two FP32 solves run the same kernels on the same grid


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ffg.build()
    ffg.load()


def _graph(spec, seed, nbh):
    f = torch.from_numpy(fi.runtimes(spec, seed)).cuda()
    return ffg.build_graph(ffg.Space.from_spec(spec), f, nbh)


@pytest.mark.parametrize("prec", [ffg.F64, ffg.F32])
def test_static_scratch_matches_workspace_entry_point(prec):
    dt = torch.float64 if prec == ffg.F64 else torch.float32
    bar = F64_L1 if prec == ffg.F64 else F32_L1
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(fi.single_small(), ffg.HAMMING), (fi.pnpoly_space(), ffg.ADJACENT),
             (fi.conv_mi50_space(), ffg.HAMMING)]
    for spec, nbh in cases:
        g = _graph(spec, 3, nbh)
        ref, it_ref, res_ref, conv = ffg.pagerank(g, 0.85, 1e-12, prec=prec)
        assert conv
        for _ in range(2):   # two calls in a row share the static scratch
            x = torch.full((g.n_nodes,), -1.0, dtype=dt, device="cuda")
            st, it, res = ffg.pagerank_solve_static(g.c, 0.85, 1e-12, 10000, prec,
                                                    x.data_ptr(), 0, stream)
            assert st == ffg.FFG_OK, ffg.ffg_last_error()
            assert it == it_ref
            l1 = float((x.double() - ref.double()).abs().sum())
            assert l1 <= bar, (spec.name, l1)
        # warm start from the converged ranks, against the same warm start
        # through the workspace entry point
        warm, it_w, _, _ = ffg.pagerank(g, 0.85, 1e-12, prec=prec, init=ref)
        x = ref.clone()
        st, it, res = ffg.pagerank_solve_static(g.c, 0.85, 1e-12, 10000, prec, x.data_ptr(),
                                                ffg.INIT_RANKS, stream)
        assert st == ffg.FFG_OK, ffg.ffg_last_error()
        assert it == it_w and it <= it_ref, (it, it_w, it_ref)
        assert float((x.double() - warm.double()).abs().sum()) <= bar


def test_static_scratch_rejects_large_graphs():
    spec = fi.single_large()
    g = _graph(spec, 1, ffg.HAMMING)
    x = torch.empty(g.n_nodes, dtype=torch.float32, device="cuda")
    st, _, _ = ffg.pagerank_solve_static(g.c, 0.85, 1e-12, 100, ffg.F32, x.data_ptr(), 0,
                                         torch.cuda.current_stream().cuda_stream)
    assert st == ffg.FFG_ERR_NO_MEMORY
    assert "static" in ffg.ffg_last_error()
