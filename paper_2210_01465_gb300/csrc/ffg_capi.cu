// ffg_capi.cu -- host-side pieces shared by every entry point: status strings,
// per-thread error detail, the launch counter and validation of a search
// space (Sec. III-B: X = S_1 x ... x S_n over integer value lists).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "ffg_internal.cuh"

namespace ffg {

std::atomic<uint64_t> g_launches{0};
static thread_local char t_error[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_error, sizeof(t_error), fmt, ap);
    va_end(ap);
}
void clear_error() { t_error[0] = '\0'; }

ffg_status check_cuda(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return FFG_OK;
    set_error("%s: %s", what, cudaGetErrorString(e));
    return FFG_ERR_CUDA;
}

ffg_status check_launch(const char *what) { return check_cuda(cudaGetLastError(), what); }

// |product| over the masked parameters of their largest |value| must fit
// int64 at every step of the running product (parameter index order).
static bool mask_product_fits(const ffg_space *s, const int64_t *maxabs, uint32_t mask) {
    unsigned __int128 p = 1;
    for (int i = 0; i < s->n_params; ++i) {
        if (!(mask & (1u << i))) continue;
        p *= (unsigned __int128)maxabs[i];
        if (p > (unsigned __int128)INT64_MAX) return false;
    }
    return true;
}

ffg_status make_dev_space(const ffg_space *s, DevSpace *d) {
    if (!s || !d) return set_error("space is NULL"), FFG_ERR_INVALID_ARG;
    if (s->n_params < 1 || s->n_params > FFG_MAX_PARAMS)
        return set_error("n_params %d outside [1,%d]", s->n_params, FFG_MAX_PARAMS),
               FFG_ERR_INVALID_ARG;
    if (!s->radix || !s->values) return set_error("radix or values is NULL"), FFG_ERR_INVALID_ARG;
    if (s->n_constraints < 0 || s->n_constraints > FFG_MAX_CONSTRAINTS ||
        (s->n_constraints > 0 && !s->constraints))
        return set_error("bad constraint list (%d)", s->n_constraints), FFG_ERR_INVALID_ARG;
    memset(d, 0, sizeof(*d));
    d->n_params = s->n_params;
    d->n_clauses = s->n_constraints;
    int64_t total_values = 0;
    for (int i = 0; i < s->n_params; ++i) {
        if (s->radix[i] < 1) return set_error("radix[%d] < 1", i), FFG_ERR_INVALID_ARG;
        total_values += s->radix[i];
        if (total_values > FFG_MAX_VALUES)
            return set_error("more than %d values in total", FFG_MAX_VALUES), FFG_ERR_INVALID_ARG;
    }
    d->n_values = (int32_t)total_values;
    int64_t R = 1;
    for (int i = 0; i < s->n_params; ++i) {
        if (R > (int64_t)INT32_MAX / s->radix[i])
            return set_error("more than 2^31-1 raw points"), FFG_ERR_OVERFLOW;
        R *= s->radix[i];
    }
    d->n_raw = R;
    int64_t off = 0, maxabs[FFG_MAX_PARAMS];
    for (int i = 0; i < s->n_params; ++i) {
        d->radix[i] = s->radix[i];
        d->voff[i] = (int32_t)off;
        maxabs[i] = 0;
        for (int j = 0; j < s->radix[i]; ++j) {
            int64_t v = s->values[off + j];
            d->values[off + j] = v;
            if (v == INT64_MIN) return set_error("value INT64_MIN not supported"), FFG_ERR_OVERFLOW;
            int64_t a = v < 0 ? -v : v;
            if (a > maxabs[i]) maxabs[i] = a;
        }
        off += s->radix[i];
    }
    int64_t st = 1;
    for (int i = s->n_params - 1; i >= 0; --i) {
        d->stride[i] = st;
        st *= s->radix[i];
    }
    const uint32_t all = (s->n_params == 32) ? 0xffffffffu : ((1u << s->n_params) - 1u);
    for (int c = 0; c < s->n_constraints; ++c) {
        const ffg_constraint &k = s->constraints[c];
        if (k.kind < FFG_PROD_LE || k.kind > FFG_PROD_LE_PROD)
            return set_error("constraint %d: unknown kind %d", c, k.kind), FFG_ERR_INVALID_ARG;
        if ((k.mask_a & ~all) || (k.mask_b & ~all) || k.reserved != 0)
            return set_error("constraint %d: mask names a missing parameter", c),
                   FFG_ERR_INVALID_ARG;
        if (!mask_product_fits(s, maxabs, k.mask_a) || !mask_product_fits(s, maxabs, k.mask_b))
            return set_error("constraint %d: product can exceed int64", c), FFG_ERR_OVERFLOW;
        d->clause[c].kind = k.kind;
        d->clause[c].mask_a = k.mask_a;
        d->clause[c].mask_b = k.mask_b;
        d->clause[c].bound = k.bound;
    }
    return FFG_OK;
}

}  // namespace ffg

extern "C" {

const char *ffg_status_str(ffg_status s) {
    switch (s) {
    case FFG_OK: return "ok";
    case FFG_ERR_INVALID_ARG: return "invalid argument";
    case FFG_ERR_OVERFLOW: return "size or product overflow";
    case FFG_ERR_CUDA: return "CUDA error";
    case FFG_ERR_EMPTY: return "empty space or no local minimum";
    case FFG_ERR_NOT_CONVERGED: return "not converged";
    case FFG_ERR_TIMEOUT: return "device wait timed out";
    case FFG_ERR_NO_MEMORY: return "workspace too small";
    }
    return "unknown status";
}

const char *ffg_last_error(void) { return ffg::t_error; }

uint64_t ffg_launch_count(void) { return ffg::g_launches.load(); }

int ffg_checked_build(void) {
#ifdef FFG_CHECKED
    return 1;
#else
    return 0;
#endif
}

uint64_t ffg_checked_failures(uint64_t *first_code, int reset) {
    using Reader = void (*)(unsigned long long *, unsigned long long *, bool);
    const Reader readers[] = {ffg::check_read_build, ffg::check_read_pagerank,
                              ffg::check_read_dag, ffg::check_read_walk,
                              ffg::check_read_centrality};
    unsigned long long total = 0, first = 0;
    for (Reader r : readers) {
        unsigned long long code = 0, count = 0;
        r(&code, &count, reset != 0);
        if (!first && code) first = code;
        total += count;
    }
    if (first_code) *first_code = first;
    return total;
}

}  // extern "C"
