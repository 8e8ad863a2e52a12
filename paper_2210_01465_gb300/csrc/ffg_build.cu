// ffg_build.cu -- construction of the fitness flow graph (Sec. VII-B) of a
// discrete tuning space (Sec. III-B) on sm_103a.
//
// One thread per raw point r, warps over 32 consecutive raw points:
//   k_valid  decodes r into mixed-radix digits, evaluates the clauses and
//            writes one 32-bit word of the validity bitmap per warp (ballot);
//            also reduces the node count and f_opt (best non-failed fitness).
//   scan     of the per-word popcounts gives the rank directory: the node id
//            of a valid raw point is prefix[r/32] + popc(word & lanes below).
//   k_count  enumerates the neighbours of every valid point -- Hamming: every
//            other value of one parameter (Eq. 2); adjacent: the list
//            neighbours d-1 and d+1 -- keeps the valid ones (bitmap) and
//            counts those with strictly lower (out) and higher (in) key.
//   scans    of the degrees give out_ptr / in_ptr.
//   k_emit   enumerates again in ascending raw order and writes node ids.
//
// Ascending raw offset order without sorting: offsets (j - d_i) * stride_i
// with j < d_i, parameters from the slowest to the fastest, then j > d_i,
// parameters from the fastest to the slowest; this is ascending because
// (r_i - 1) * stride_i < stride_{i-1}.  Node ids are monotone in raw index,
// so the lists come out sorted by node id.
//
// For a warp of 32 consecutive raw points, the candidates for one (i, j)
// are 32 shifted consecutive raw points, so the fitness and bitmap loads of
// the enumeration are coalesced.
#include "ffg_internal.cuh"

namespace ffg {

namespace {

constexpr int kThreads = 256;

struct BuildCtl {
    unsigned long long fopt_bits;  // ordered bits of the best non-failed fitness
    unsigned long long n_nodes;
    unsigned long long n_out;      // sum of out-degrees
    unsigned long long n_in;       // sum of in-degrees
    unsigned long long n_minima;
};

struct BuildWs {
    BuildCtl *ctl;
    uint32_t *bitmap;
    int32_t *wcount;
    int64_t *wprefix;
    int32_t *outdeg;
    int32_t *indeg;
    int64_t *scratch;
    size_t bytes;
};

BuildWs carve(void *base, int64_t R) {
    const int64_t W = (R + 31) / 32;
    Carver c(base);
    BuildWs w;
    w.ctl = c.take<BuildCtl>(1);
    w.bitmap = c.take<uint32_t>(W);
    w.wcount = c.take<int32_t>(W);
    w.wprefix = c.take<int64_t>(W + 1);
    w.outdeg = c.take<int32_t>(R);
    w.indeg = c.take<int32_t>(R);
    w.scratch = c.take<int64_t>(scan_scratch_elems(R > W ? R : W));
    w.bytes = c.off;
    return w;
}

// the parts of the space a block needs, staged in shared memory
struct SmemSpace {
    int32_t n, nc;
    int32_t radix[FFG_MAX_PARAMS];
    int32_t voff[FFG_MAX_PARAMS];
    uint32_t stride[FFG_MAX_PARAMS];
    DevClause clause[FFG_MAX_CONSTRAINTS];
};

__device__ __forceinline__ void stage_space(const DevSpace &sp, SmemSpace &s, int64_t *vals,
                                            bool with_values) {
    const int t = threadIdx.x;
    if (t == 0) {
        s.n = sp.n_params;
        s.nc = sp.n_clauses;
    }
    if (t < FFG_MAX_PARAMS) {
        s.radix[t] = sp.radix[t];
        s.voff[t] = sp.voff[t];
        s.stride[t] = static_cast<uint32_t>(sp.stride[t]);
    }
    if (t < FFG_MAX_CONSTRAINTS) s.clause[t] = sp.clause[t];
    if (with_values)
        for (int i = t; i < sp.n_values; i += blockDim.x) vals[i] = sp.values[i];
    __syncthreads();
}

__device__ __forceinline__ bool bit_of(const uint32_t *__restrict__ bm, uint32_t r) {
    return (__ldg(bm + (r >> 5)) >> (r & 31)) & 1u;
}

__device__ __forceinline__ int32_t rank_of(const uint32_t *__restrict__ bm,
                                           const int64_t *__restrict__ wprefix, uint32_t r) {
    const uint32_t w = __ldg(bm + (r >> 5));
    return static_cast<int32_t>(__ldg(wprefix + (r >> 5)) + __popc(w & ((1u << (r & 31)) - 1u)));
}

template <typename T>
__device__ __forceinline__ T block_sum(T v) {
    __shared__ T red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    T s = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    return s;  // valid in thread 0
}

__device__ __forceinline__ unsigned long long block_min_u64(unsigned long long v) {
    __shared__ unsigned long long red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(0xffffffffu, v, o);
        v = t < v ? t : v;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    unsigned long long m = ~0ULL;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = red[k] < m ? red[k] : m;
    return m;
}

__device__ __forceinline__ int64_t mask_product(const SmemSpace &s, const int64_t *vals,
                                                const int32_t *digit, uint32_t mask) {
    int64_t p = 1;
    while (mask) {
        const int i = __ffs(mask) - 1;
        mask &= mask - 1;
        p *= vals[s.voff[i] + digit[i]];
    }
    return p;
}

// ---------------------------------------------------------------------------
// k_valid: validity bitmap, per-word counts, node count, f_opt
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_valid(const DevSpace sp,
                                                    const double *__restrict__ fit,
                                                    double fail_thr, uint32_t *__restrict__ bitmap,
                                                    int32_t *__restrict__ wcount, BuildCtl *ctl) {
    __shared__ SmemSpace s;
    __shared__ int64_t vals[FFG_MAX_VALUES];
    stage_space(sp, s, vals, true);
    const int64_t R = sp.n_raw;
    const int64_t W = (R + 31) >> 5;
    const int64_t r = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    bool ok = false;
    unsigned long long fbits = ~0ULL;
    if (r < R) {
        int32_t digit[FFG_MAX_PARAMS];
        uint32_t rem = static_cast<uint32_t>(r);
        for (int i = s.n - 1; i >= 0; --i) {
            const uint32_t q = rem / static_cast<uint32_t>(s.radix[i]);
            digit[i] = static_cast<int32_t>(rem - q * static_cast<uint32_t>(s.radix[i]));
            rem = q;
        }
        ok = true;
        for (int c = 0; c < s.nc; ++c) {
            const DevClause &cl = s.clause[c];
            const int64_t pa = mask_product(s, vals, digit, cl.mask_a);
            const int64_t pb = mask_product(s, vals, digit, cl.mask_b);
            bool h;
            switch (cl.kind) {
            case FFG_PROD_LE: h = pa <= cl.bound; break;
            case FFG_PROD_GE: h = pa >= cl.bound; break;
            case FFG_DIVIDES: h = (pb != 0) && (pa % pb == 0); break;
            default: h = pa <= pb; break;
            }
            ok = ok && h;
        }
        if (ok) {
            const double f = fit[r];
            if (f < fail_thr) fbits = ordered_bits(f);
        }
    }
    const unsigned m = __ballot_sync(0xffffffffu, ok);
    if ((threadIdx.x & 31) == 0 && (r >> 5) < W) {
        bitmap[r >> 5] = m;
        wcount[r >> 5] = __popc(m);
    }
    const unsigned long long cnt = block_sum<unsigned long long>(ok ? 1ULL : 0ULL);
    const unsigned long long fmin = block_min_u64(fbits);
    if (threadIdx.x == 0) {
        if (cnt) atomicAdd(&ctl->n_nodes, cnt);
        if (fmin != ~0ULL) atomicMin(&ctl->fopt_bits, fmin);
    }
}

// ---------------------------------------------------------------------------
// k_count: out/in degree of every node
// ---------------------------------------------------------------------------
template <int NBH>
__global__ void __launch_bounds__(kThreads) k_count(const DevSpace sp,
                                                    const double *__restrict__ fit,
                                                    double fail_thr,
                                                    const uint32_t *__restrict__ bitmap,
                                                    const int64_t *__restrict__ wprefix,
                                                    int32_t *__restrict__ outdeg,
                                                    int32_t *__restrict__ indeg, BuildCtl *ctl) {
    __shared__ SmemSpace s;
    stage_space(sp, s, nullptr, false);
    const int64_t R = sp.n_raw;
    const int64_t r64 = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    unsigned long long n_out = 0, n_in = 0, n_min = 0;
    if (r64 < R && bit_of(bitmap, static_cast<uint32_t>(r64))) {
        const uint32_t r = static_cast<uint32_t>(r64);
        const double k0 = fit_key(__ldg(fit + r), fail_thr);
        int32_t out = 0, in = 0;
        uint32_t rem = r;
        for (int i = s.n - 1; i >= 0; --i) {
            const uint32_t rad = static_cast<uint32_t>(s.radix[i]);
            const uint32_t q = rem / rad;
            const uint32_t d = rem - q * rad;
            rem = q;
            const uint32_t st = s.stride[i];
            const uint32_t base = r - d * st;
            const uint32_t jlo = NBH == FFG_HAMMING ? 0u : (d > 0 ? d - 1 : 0u);
            const uint32_t jhi = NBH == FFG_HAMMING ? rad - 1 : (d + 1 < rad ? d + 1 : d);
            for (uint32_t j = jlo; j <= jhi; ++j) {
                if (j == d) continue;
                const uint32_t rr = base + j * st;
                if (!bit_of(bitmap, rr)) continue;
                const double kk = fit_key(__ldg(fit + rr), fail_thr);
                out += kk < k0;
                in += kk > k0;
            }
        }
        const int32_t node = rank_of(bitmap, wprefix, r);
        outdeg[node] = out;
        indeg[node] = in;
        n_out = out;
        n_in = in;
        n_min = (k0 < fail_thr && out == 0) ? 1 : 0;
    }
    const unsigned long long so = block_sum(n_out);
    const unsigned long long si = block_sum(n_in);
    const unsigned long long sm = block_sum(n_min);
    if (threadIdx.x == 0) {
        if (so) atomicAdd(&ctl->n_out, so);
        if (si) atomicAdd(&ctl->n_in, si);
        if (sm) atomicAdd(&ctl->n_minima, sm);
    }
}

// ---------------------------------------------------------------------------
// k_emit: canonical CSR rows, outdeg, node_raw, is_min
// ---------------------------------------------------------------------------
template <int NBH>
__global__ void __launch_bounds__(kThreads) k_emit(
    const DevSpace sp, const double *__restrict__ fit, double fail_thr,
    const uint32_t *__restrict__ bitmap, const int64_t *__restrict__ wprefix,
    const int64_t *__restrict__ out_ptr, const int64_t *__restrict__ in_ptr,
    int32_t *__restrict__ out_idx, int32_t *__restrict__ in_idx, int32_t *__restrict__ outdeg,
    int64_t *__restrict__ node_raw, uint8_t *__restrict__ is_min) {
    __shared__ SmemSpace s;
    stage_space(sp, s, nullptr, false);
    const int64_t R = sp.n_raw;
    const int64_t r64 = int64_t(blockIdx.x) * kThreads + threadIdx.x;
    if (r64 >= R || !bit_of(bitmap, static_cast<uint32_t>(r64))) return;
    const uint32_t r = static_cast<uint32_t>(r64);
    const double k0 = fit_key(__ldg(fit + r), fail_thr);
    const int32_t node = rank_of(bitmap, wprefix, r);
    const int64_t o0 = out_ptr[node];
    int64_t o = o0, q = in_ptr[node];

    uint32_t digit[FFG_MAX_PARAMS];
    {
        uint32_t rem = r;
#pragma unroll
        for (int i = FFG_MAX_PARAMS - 1; i >= 0; --i) {
            if (i < s.n) {
                const uint32_t rad = static_cast<uint32_t>(s.radix[i]);
                const uint32_t qq = rem / rad;
                digit[i] = rem - qq * rad;
                rem = qq;
            }
        }
    }
    auto visit = [&](uint32_t rr) {
        if (!bit_of(bitmap, rr)) return;
        const double kk = fit_key(__ldg(fit + rr), fail_thr);
        if (kk < k0) out_idx[o++] = rank_of(bitmap, wprefix, rr);
        else if (kk > k0) in_idx[q++] = rank_of(bitmap, wprefix, rr);
    };
    // negative offsets: slowest parameter first, values ascending
#pragma unroll
    for (int i = 0; i < FFG_MAX_PARAMS; ++i) {
        if (i < s.n) {
            const uint32_t d = digit[i], st = s.stride[i];
            const uint32_t jlo = NBH == FFG_HAMMING ? 0u : (d > 0 ? d - 1 : 0u);
            for (uint32_t j = jlo; j < d; ++j) visit(r - (d - j) * st);
        }
    }
    // positive offsets: fastest parameter first, values ascending
#pragma unroll
    for (int i = FFG_MAX_PARAMS - 1; i >= 0; --i) {
        if (i < s.n) {
            const uint32_t d = digit[i], st = s.stride[i];
            const uint32_t rad = static_cast<uint32_t>(s.radix[i]);
            const uint32_t jhi = NBH == FFG_HAMMING ? rad : (d + 2 < rad ? d + 2 : rad);
            for (uint32_t j = d + 1; j < jhi; ++j) visit(r + (j - d) * st);
        }
    }
    const int32_t od = static_cast<int32_t>(o - o0);
    outdeg[node] = od;
    node_raw[node] = r;
    is_min[node] = (k0 < fail_thr && od == 0) ? 1 : 0;
}

ffg_status check_common(const ffg_space *space, const double *fitness_raw, ffg_nbh nbh,
                        double fail_thr, const ffg_graph *g, void *ws, DevSpace *d,
                        BuildWs *w, size_t ws_bytes) {
    FFG_TRY(make_dev_space(space, d));
    if (nbh != FFG_HAMMING && nbh != FFG_ADJACENT)
        return set_error("unknown neighbourhood %d", (int)nbh), FFG_ERR_INVALID_ARG;
    if (!fitness_raw || !g || !ws)
        return set_error("fitness_raw, graph and workspace must be non-NULL"),
               FFG_ERR_INVALID_ARG;
    if (fail_thr != fail_thr) return set_error("fail_thr is NaN"), FFG_ERR_INVALID_ARG;
    if (!aligned256(ws)) return set_error("workspace not 256-byte aligned"), FFG_ERR_INVALID_ARG;
    *w = carve(ws, d->n_raw);
    if (ws_bytes < w->bytes)
        return set_error("workspace %zu bytes, need %zu", ws_bytes, w->bytes), FFG_ERR_NO_MEMORY;
    return FFG_OK;
}

}  // namespace

}  // namespace ffg

using namespace ffg;

extern "C" size_t ffg_workspace_bytes(const ffg_space *space, ffg_nbh nbh) {
    (void)nbh;
    DevSpace d;
    if (make_dev_space(space, &d) != FFG_OK) return 0;
    return carve(nullptr, d.n_raw).bytes;
}

extern "C" ffg_status ffg_build_count(const ffg_space *space, const double *fitness_raw,
                                      ffg_nbh nbh, double fail_thr, ffg_graph *g,
                                      int64_t *n_nodes, int64_t *n_edges, void *workspace,
                                      size_t ws_bytes, void *stream_) {
    clear_error();
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    DevSpace d;
    BuildWs w;
    FFG_TRY(check_common(space, fitness_raw, nbh, fail_thr, g, workspace, &d, &w, ws_bytes));
    const int64_t R = d.n_raw, W = (R + 31) / 32;
    const unsigned grid = static_cast<unsigned>((R + kThreads - 1) / kThreads);
    FFG_TRY(check_cuda(cudaMemsetAsync(w.ctl, 0, sizeof(BuildCtl), stream), "memset"));
    FFG_TRY(check_cuda(cudaMemsetAsync(&w.ctl->fopt_bits, 0xff, 8, stream), "memset"));
    k_valid<<<grid, kThreads, 0, stream>>>(d, fitness_raw, fail_thr, w.bitmap, w.wcount, w.ctl);
    count_launch();
    FFG_TRY(check_launch("k_valid"));
    FFG_TRY(scan_exclusive(w.wcount, w.wprefix, W, w.scratch, stream));
    if (nbh == FFG_HAMMING)
        k_count<FFG_HAMMING><<<grid, kThreads, 0, stream>>>(d, fitness_raw, fail_thr, w.bitmap,
                                                            w.wprefix, w.outdeg, w.indeg, w.ctl);
    else
        k_count<FFG_ADJACENT><<<grid, kThreads, 0, stream>>>(d, fitness_raw, fail_thr, w.bitmap,
                                                             w.wprefix, w.outdeg, w.indeg, w.ctl);
    count_launch();
    FFG_TRY(check_launch("k_count"));
    BuildCtl h;
    FFG_TRY(check_cuda(cudaMemcpyAsync(&h, w.ctl, sizeof(h), cudaMemcpyDeviceToHost, stream),
                       "read counts"));
    FFG_TRY(check_cuda(cudaStreamSynchronize(stream), "sync counts"));
    if (h.n_out != h.n_in) {
        set_error("internal: out-degree sum %llu != in-degree sum %llu", h.n_out, h.n_in);
        return FFG_ERR_CUDA;
    }
    g->n_raw = R;
    g->n_nodes = static_cast<int64_t>(h.n_nodes);
    g->n_edges = static_cast<int64_t>(h.n_out);
    g->n_minima = static_cast<int64_t>(h.n_minima);
    g->f_opt = h.fopt_bits == ~0ULL ? __builtin_inf() : from_ordered_bits(h.fopt_bits);
    if (n_nodes) *n_nodes = g->n_nodes;
    if (n_edges) *n_edges = g->n_edges;
    if (g->n_nodes == 0) return set_error("no valid configuration"), FFG_ERR_EMPTY;
    return FFG_OK;
}

extern "C" ffg_status ffg_build_fill(const ffg_space *space, const double *fitness_raw,
                                     ffg_nbh nbh, double fail_thr, ffg_graph *g, void *workspace,
                                     size_t ws_bytes, void *stream_) {
    clear_error();
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    DevSpace d;
    BuildWs w;
    FFG_TRY(check_common(space, fitness_raw, nbh, fail_thr, g, workspace, &d, &w, ws_bytes));
    if (g->n_raw != d.n_raw || g->n_nodes <= 0 || g->n_nodes > d.n_raw || g->n_edges < 0)
        return set_error("graph sizes do not come from ffg_build_count"), FFG_ERR_INVALID_ARG;
    if (!g->out_ptr || !g->in_ptr || !g->outdeg || !g->node_raw || !g->is_min ||
        (g->n_edges > 0 && (!g->out_idx || !g->in_idx)))
        return set_error("a graph buffer is NULL"), FFG_ERR_INVALID_ARG;
    const int64_t R = d.n_raw, N = g->n_nodes;
    const unsigned grid = static_cast<unsigned>((R + kThreads - 1) / kThreads);
    FFG_TRY(scan_exclusive(w.outdeg, g->out_ptr, N, w.scratch, stream));
    FFG_TRY(scan_exclusive(w.indeg, g->in_ptr, N, w.scratch, stream));
    if (nbh == FFG_HAMMING)
        k_emit<FFG_HAMMING><<<grid, kThreads, 0, stream>>>(
            d, fitness_raw, fail_thr, w.bitmap, w.wprefix, g->out_ptr, g->in_ptr, g->out_idx,
            g->in_idx, g->outdeg, g->node_raw, g->is_min);
    else
        k_emit<FFG_ADJACENT><<<grid, kThreads, 0, stream>>>(
            d, fitness_raw, fail_thr, w.bitmap, w.wprefix, g->out_ptr, g->in_ptr, g->out_idx,
            g->in_idx, g->outdeg, g->node_raw, g->is_min);
    count_launch();
    return check_launch("k_emit");
}
