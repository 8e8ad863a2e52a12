// ffg_batch.cu -- ffg_batch_run: one call that re-runs a planned batch of
// search spaces end to end -- every FFG, every PageRank solve and every
// proportion of centrality (Sec. VII-B, Eq. 3, over many spaces at once).
// It only sequences the batched entry points; the work is theirs.
#include <string>
#include <vector>

#include "ffg_internal.cuh"

using namespace ffg;

namespace {

// keeps the first failure's status and detail; a CUDA error or a timeout
// outranks every other status
struct Worst {
    ffg_status st = FFG_OK;
    std::string detail;
    void add(ffg_status s) {
        if (s == FFG_OK) return;
        const bool severe = s == FFG_ERR_CUDA || s == FFG_ERR_TIMEOUT;
        const bool held_severe = st == FFG_ERR_CUDA || st == FFG_ERR_TIMEOUT;
        if (st == FFG_OK || (severe && !held_severe)) {
            st = s;
            detail = ffg_last_error();
        }
    }
};

}  // namespace

extern "C" ffg_status ffg_batch_run(const ffg_batch_desc *d, ffg_batch_out *out,
                                    void *stream) {
    clear_error();
    if (!d || !d->pagerank || d->pagerank->n_jobs < 1)
        return set_error("desc and a planned pagerank batch are required"), FFG_ERR_INVALID_ARG;
    if (d->build && d->build->n_jobs < 1)
        return set_error("build plan is empty"), FFG_ERR_INVALID_ARG;
    if (d->cp && d->cp->n_jobs < 1) return set_error("C_p plan is empty"), FFG_ERR_INVALID_ARG;
    if (out && out->cp && !d->cp)
        return set_error("out->cp needs a C_p plan (desc->cp)"), FFG_ERR_INVALID_ARG;

    // launches only: the graphs, every solve, every C_p
    if (d->build) FFG_TRY(ffg_build_batch_rerun(d->build, stream));
    FFG_TRY(pagerank_batch_run(d->pagerank, stream));
    if (d->cp) FFG_TRY(centrality_batch_run(d->cp, stream));
    if (!out) return FFG_OK;

    Worst w;
    if (d->build) {
        std::vector<int32_t> own;
        int32_t *st = out->build_status;
        if (!st) {
            own.resize(size_t(d->build->n_jobs));
            st = own.data();
        }
        w.add(ffg_build_batch_query(d->build, st, stream));
        if (w.st == FFG_ERR_CUDA) return set_error("%s", w.detail.c_str()), w.st;
    }
    w.add(pagerank_batch_query(d->pagerank, out->iters, out->residual, out->pr_status, stream));
    if (w.st == FFG_ERR_CUDA || w.st == FFG_ERR_TIMEOUT)
        return set_error("%s", w.detail.c_str()), w.st;
    if (d->cp) w.add(centrality_batch_query(d->cp, out->cp, nullptr, stream));
    if (w.st != FFG_OK) set_error("%s", w.detail.c_str());
    return w.st;
}
