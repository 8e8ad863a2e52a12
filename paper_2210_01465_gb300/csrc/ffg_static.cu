// ffg_static.cu -- pagerank_solve_static: PageRank whose scratch space is a
// file-scope device array instead of a caller-provided workspace.
#include "ffg_internal.cuh"

using namespace ffg;

// ---------------------------------------------------------------------------
// PageRank without a caller-provided workspace.
//
// Some callers cannot allocate device memory when they want centralities:
// code that runs while another component owns all device memory through its
// own pool, or that runs where cudaMalloc is not allowed or would stall the
// device (it can synchronise), e.g. a tuning loop embedded in a
// latency-sensitive application.  For them the scratch space lives in one
// file-scope device array, allocated when the library is loaded on a device
// and held until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticScratchBytes = size_t(8) << 20;  // 8 MiB per device
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch on the current device.  The host-side
// symbol is not a device address.  The lookup is repeated on every call: it
// is cheap next to the synchronising solve, and the address can change when
// the device's primary context is reset and the module loaded again.  The
// first lookup on a device loads the library's module there, which must not
// happen inside a stream capture.
ffg_status static_scratch(void **out) {
    void *p = nullptr;
    FFG_TRY(check_cuda(cudaGetSymbolAddress(&p, g_static_scratch),
                       "cudaGetSymbolAddress(static scratch)"));
    *out = p;
    return FFG_OK;
}

}  // namespace

extern "C" ffg_status pagerank_solve_static(const ffg_graph *g, double damping, double tol,
                                            int32_t max_iter, ffg_prec prec, void *ranks,
                                            int init, int32_t *iters_out, double *residual_out,
                                            void *stream) {
    clear_error();
    if (!g || g->n_nodes <= 0 || g->n_edges < 0)
        return set_error("graph is empty or incomplete"), FFG_ERR_INVALID_ARG;
    if (init & ~(FFG_INIT_RANKS | FFG_INIT_LAYOUT))
        return set_error("unknown init flags 0x%x", init), FFG_ERR_INVALID_ARG;
    const size_t need = pagerank_workspace_bytes(g->n_nodes, g->n_edges, prec);
    if (need > kStaticScratchBytes) {
        set_error("pagerank_solve_static: this graph needs %zu bytes of scratch, the static "
                  "scratch holds %zu; use pagerank_solve with a workspace",
                  need, kStaticScratchBytes);
        return FFG_ERR_NO_MEMORY;
    }
    void *scratch = nullptr;
    FFG_TRY(static_scratch(&scratch));
    int32_t iters = 0;
    double res = 0.0;
    // the static scratch never holds a prepared layout of the caller's graph
    const ffg_status st = pagerank_solve(g, damping, tol, max_iter, prec, ranks,
                                         init & FFG_INIT_RANKS, scratch, kStaticScratchBytes,
                                         &iters, &res, stream);
    if (iters_out) *iters_out = iters;
    if (residual_out) *residual_out = res;
    return st;
}
