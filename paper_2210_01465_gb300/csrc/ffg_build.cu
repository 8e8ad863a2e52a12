// ffg_build.cu -- construction of the fitness flow graph (Sec. VII-B) of a
// discrete tuning space (Sec. III-B) on sm_103a.
//
// One thread per raw point r, warps over 32 consecutive raw points:
//   k_valid  decodes r into mixed-radix digits, evaluates the clauses and
//            writes one 32-bit word of the validity bitmap per warp (ballot)
//            and the point's key: the fitness (+inf if failed) as an
//            order-preserving 64-bit integer, 0 if invalid, so that the
//            enumerations compare integers -- a warp-wide FP64 compare
//            occupies an SM's narrow FP64 units on this part -- and an
//            invalid neighbour fails both comparisons without a separate
//            test; also reduces the node count and f_opt (best non-failed
//            fitness).
//   scan     of the per-word popcounts gives the rank directory: the node id
//            of a valid raw point is prefix[r/32] + popc(word & lanes below).
//   k_nodes  records every valid point's node id and the node list (raw
//            point of every node), so that the enumerations below run one
//            thread per node: no lane idles on an invalid point.
//   k_count  enumerates the neighbours of every node -- Hamming: every
//            other value of one parameter (Eq. 2); adjacent: the list
//            neighbours d-1 and d+1 -- and counts those with strictly lower
//            (out) and higher (in) key.
//   scans    of the degrees give out_ptr / in_ptr.
//   k_emit   enumerates again in ascending raw order and writes node ids.
//
// Ascending raw offset order without sorting: offsets (j - d_i) * stride_i
// with j < d_i, parameters from the slowest to the fastest, then j > d_i,
// parameters from the fastest to the slowest; this is ascending because
// (r_i - 1) * stride_i < stride_{i-1}.  Node ids are monotone in raw index,
// so the lists come out sorted by node id.
//
// For a warp of 32 consecutive nodes, the candidates for one (i, j) are
// shifted nearly consecutive raw points, so the key and node-id loads of the
// enumeration are close to coalesced.  Digits come from divisions by the radices done
// as one multiply-high each (Lemire, Kaser and Kurz 2019: for 32-bit n and
// d >= 2, floor(n / d) = (n * ceil(2^64 / d)) >> 64).
#include <vector>

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
    unsigned long long *key;  // per raw point: ordered fitness key, 0 if invalid
    int32_t *node_of;  // per valid raw point: node id
    int32_t *nodes;    // per node: its raw point
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
    w.key = c.take<unsigned long long>(R);
    w.node_of = c.take<int32_t>(R);
    w.nodes = c.take<int32_t>(R);
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
    unsigned long long magic[FFG_MAX_PARAMS];  // ceil(2^64 / radix), radix >= 2
    DevClause clause[FFG_MAX_CONSTRAINTS];
};

// n / radix_i for n < 2^31
__device__ __forceinline__ uint32_t div_radix(const SmemSpace &s, int i, uint32_t n) {
    return s.radix[i] == 1 ? n : static_cast<uint32_t>(__umul64hi(n, s.magic[i]));
}

// Keys: fit_key (failed points +inf) mapped by ordered_bits, which is
// monotone and never 0 for a non-NaN double, so 0 marks an invalid point;
// -0 is first made +0 (the two compare equal).  For valid keys a and b,
// a < b as integers iff a < b as doubles; with the 0 of an invalid point,
// (a - 1 < b - 1) and (a > b) are both false.
constexpr unsigned long long kInvalidKey = 0ULL;
constexpr unsigned long long kFailedKey = 0xfff0000000000000ULL;  // ordered_bits(+inf)
__device__ __forceinline__ unsigned long long key_of(double f, double fail_thr) {
    const double k = fit_key(f, fail_thr);
    return ordered_bits(k == 0.0 ? 0.0 : k);
}
__device__ __forceinline__ bool key_below(unsigned long long a, unsigned long long b) {
    return a - 1ULL < b - 1ULL;  // a < b, false when a is invalid
}

__device__ __forceinline__ void stage_space(const DevSpace &sp, SmemSpace &s, int64_t *vals,
                                            bool with_values) {
    const int t = threadIdx.x;
    if (t == 0) {
        s.n = sp.n_params;
        s.nc = sp.n_clauses;
    }
    if (t < FFG_MAX_PARAMS) {
        const int32_t r = sp.radix[t];
        s.radix[t] = r;
        s.voff[t] = sp.voff[t];
        s.stride[t] = static_cast<uint32_t>(sp.stride[t]);
        s.magic[t] = r >= 2 ? ~0ULL / static_cast<unsigned long long>(r) + 1ULL : 0ULL;
    }
    if (t < FFG_MAX_CONSTRAINTS) s.clause[t] = sp.clause[t];
    if (with_values)
        for (int i = t; i < sp.n_values; i += blockDim.x) vals[i] = sp.values[i];
    __syncthreads();
}

// node id of valid raw point r; wprefix may be a slice of a longer scan
// whose value at the space's first word is wbase
__device__ __forceinline__ int32_t rank_of(const uint32_t *__restrict__ bm,
                                           const int64_t *__restrict__ wprefix, int64_t wbase,
                                           uint32_t r) {
    const uint32_t w = __ldg(bm + (r >> 5));
    return static_cast<int32_t>(__ldg(wprefix + (r >> 5)) - wbase +
                                __popc(w & ((1u << (r & 31)) - 1u)));
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
// validity bitmap, per-word counts, node count, f_opt (raw point r, one
// block: the space staged in s / vals)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void valid_body(const SmemSpace &s, const int64_t *vals, int64_t R,
                                           int64_t r, const double *__restrict__ fit,
                                           double fail_thr, uint32_t *__restrict__ bitmap,
                                           int32_t *__restrict__ wcount,
                                           unsigned long long *__restrict__ key,
                                           BuildCtl *ctl) {
    const int64_t W = (R + 31) >> 5;
    bool ok = false;
    unsigned long long fbits = ~0ULL;
    if (r < R) {
        int32_t digit[FFG_MAX_PARAMS];
        uint32_t rem = static_cast<uint32_t>(r);
        for (int i = s.n - 1; i >= 0; --i) {
            const uint32_t q = div_radix(s, i, rem);
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
        unsigned long long k = kInvalidKey;
        if (ok) {
            const double f = fit[r];
            if (f < fail_thr) fbits = ordered_bits(f);
            k = key_of(f, fail_thr);
        }
        key[r] = k;
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

__global__ void __launch_bounds__(kThreads) k_valid(const DevSpace sp,
                                                    const double *__restrict__ fit,
                                                    double fail_thr, uint32_t *__restrict__ bitmap,
                                                    int32_t *__restrict__ wcount,
                                                    unsigned long long *__restrict__ key,
                                                    BuildCtl *ctl) {
    __shared__ SmemSpace s;
    __shared__ int64_t vals[FFG_MAX_VALUES];
    stage_space(sp, s, vals, true);
    valid_body(s, vals, sp.n_raw, int64_t(blockIdx.x) * kThreads + threadIdx.x, fit, fail_thr,
               bitmap, wcount, key, ctl);
}

// ---------------------------------------------------------------------------
// out/in degree of every node
// ---------------------------------------------------------------------------
// node id and node list of every valid raw point (raw point r, one block)
__device__ __forceinline__ void nodes_body(int64_t R, int64_t r64,
                                           const unsigned long long *__restrict__ key,
                                           const uint32_t *__restrict__ bitmap,
                                           const int64_t *__restrict__ wprefix, int64_t wbase,
                                           int32_t *__restrict__ node_of,
                                           int32_t *__restrict__ nodes) {
    if (r64 >= R) return;
    if (__ldg(key + r64) == kInvalidKey) return;  // not a valid point
    const uint32_t r = static_cast<uint32_t>(r64);
    const int32_t node = rank_of(bitmap, wprefix, wbase, r);
    node_of[r] = node;
    nodes[node] = static_cast<int32_t>(r);
}

__global__ void __launch_bounds__(kThreads) k_nodes(int64_t R,
                                                    const unsigned long long *__restrict__ key,
                                                    const uint32_t *__restrict__ bitmap,
                                                    const int64_t *__restrict__ wprefix,
                                                    int32_t *__restrict__ node_of,
                                                    int32_t *__restrict__ nodes) {
    nodes_body(R, int64_t(blockIdx.x) * kThreads + threadIdx.x, key, bitmap, wprefix, 0, node_of,
               nodes);
}

// out/in degree of node `node` (one thread per node; nodes >= N idle)
template <int NBH>
__device__ __forceinline__ void count_body(const SmemSpace &s, int64_t R, int64_t N, int64_t node,
                                           const int32_t *__restrict__ nodes,
                                           const unsigned long long *__restrict__ key,
                                           int32_t *__restrict__ outdeg,
                                           int32_t *__restrict__ indeg, BuildCtl *ctl) {
    unsigned long long n_out = 0, n_in = 0, n_min = 0;
    if (node < N) {
        const uint32_t r = static_cast<uint32_t>(__ldg(nodes + node));
        const unsigned long long k0 = __ldg(key + r);
        int32_t out = 0, in = 0;
        uint32_t rem = r;
        for (int i = s.n - 1; i >= 0; --i) {
            const uint32_t rad = static_cast<uint32_t>(s.radix[i]);
            const uint32_t q = div_radix(s, i, rem);
            const uint32_t d = rem - q * rad;
            rem = q;
            const uint32_t st = s.stride[i];
            const uint32_t base = r - d * st;
            const uint32_t jlo = NBH == FFG_HAMMING ? 0u : (d > 0 ? d - 1 : 0u);
            const uint32_t jhi = NBH == FFG_HAMMING ? rad - 1 : (d + 1 < rad ? d + 1 : d);
            for (uint32_t j = jlo; j <= jhi; ++j) {
                if (j == d) continue;
                const uint32_t rr = base + j * st;
                const unsigned long long kk =
                    FFG_CHECK(rr < R, 203) ? __ldg(key + rr) : kInvalidKey;  // 0 if invalid
                out += key_below(kk, k0);
                in += kk > k0;
            }
        }
        outdeg[node] = out;
        indeg[node] = in;
        n_out = out;
        n_in = in;
        n_min = (k0 != kFailedKey && out == 0) ? 1 : 0;
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

// one thread per node; the node count comes from the device (blocks beyond
// it have nothing to do)
template <int NBH>
__global__ void __launch_bounds__(kThreads) k_count(const DevSpace sp,
                                                    const int32_t *__restrict__ nodes,
                                                    const unsigned long long *__restrict__ key,
                                                    int32_t *__restrict__ outdeg,
                                                    int32_t *__restrict__ indeg, BuildCtl *ctl) {
    const int64_t N = static_cast<int64_t>(*(volatile unsigned long long *)&ctl->n_nodes);
    if (int64_t(blockIdx.x) * kThreads >= N) return;  // uniform over the block
    __shared__ SmemSpace s;
    stage_space(sp, s, nullptr, false);
    count_body<NBH>(s, sp.n_raw, N, int64_t(blockIdx.x) * kThreads + threadIdx.x, nodes, key,
                    outdeg, indeg, ctl);
}

// ---------------------------------------------------------------------------
// canonical CSR rows, outdeg, node_raw, is_min
// ---------------------------------------------------------------------------
// The CSR rows of node `node` (one thread per node).
template <int NBH>
__device__ __forceinline__ void emit_body(
    const SmemSpace &s, int64_t R, int64_t N, int64_t node64, const int32_t *__restrict__ nodes,
    const unsigned long long *__restrict__ key, const int32_t *__restrict__ node_of,
    const int64_t *__restrict__ out_ptr, const int64_t *__restrict__ in_ptr,
    int32_t *__restrict__ out_idx, int32_t *__restrict__ in_idx, int32_t *__restrict__ outdeg,
    int64_t *__restrict__ node_raw, uint8_t *__restrict__ is_min) {
    if (node64 >= N) return;
    const int32_t node = static_cast<int32_t>(node64);
    const uint32_t r = static_cast<uint32_t>(__ldg(nodes + node));
    const unsigned long long k0 = __ldg(key + r);
    const int64_t o0 = out_ptr[node];
    [[maybe_unused]] const int64_t o1 = out_ptr[node + 1], q1 = in_ptr[node + 1];  // checks
    int64_t o = o0, q = in_ptr[node];

    uint32_t digit[FFG_MAX_PARAMS];
    {
        uint32_t rem = r;
#pragma unroll
        for (int i = FFG_MAX_PARAMS - 1; i >= 0; --i) {
            if (i < s.n) {
                const uint32_t rad = static_cast<uint32_t>(s.radix[i]);
                const uint32_t qq = div_radix(s, i, rem);
                digit[i] = rem - qq * rad;
                rem = qq;
            }
        }
    }
    auto visit = [&](uint32_t rr) {
        // the key and the node id load together (the node id is used only
        // for an edge, but loading it unconditionally keeps the two loads
        // independent instead of chaining a second latency per edge)
        if (!FFG_CHECK(rr < R, 203)) return;
        const unsigned long long kk = __ldg(key + rr);  // 0 if invalid: both tests false
        const int32_t id = __ldg(node_of + rr);
        if (key_below(kk, k0)) {
            if (FFG_CHECK(o < o1 && id >= 0 && id < N, 201)) out_idx[o] = id;
            ++o;
        } else if (kk > k0) {
            if (FFG_CHECK(q < q1 && id >= 0 && id < N, 202)) in_idx[q] = id;
            ++q;
        }
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
    is_min[node] = (k0 != kFailedKey && od == 0) ? 1 : 0;
}

template <int NBH>
__global__ void __launch_bounds__(kThreads) k_emit(
    const DevSpace sp, int64_t N, const int32_t *__restrict__ nodes,
    const unsigned long long *__restrict__ key, const int32_t *__restrict__ node_of,
    const int64_t *__restrict__ out_ptr, const int64_t *__restrict__ in_ptr,
    int32_t *__restrict__ out_idx, int32_t *__restrict__ in_idx, int32_t *__restrict__ outdeg,
    int64_t *__restrict__ node_raw, uint8_t *__restrict__ is_min) {
    __shared__ SmemSpace s;
    stage_space(sp, s, nullptr, false);
    emit_body<NBH>(s, sp.n_raw, N, int64_t(blockIdx.x) * kThreads + threadIdx.x, nodes, key,
                   node_of, out_ptr, in_ptr, out_idx, in_idx, outdeg, node_raw, is_min);
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
    k_valid<<<grid, kThreads, 0, stream>>>(d, fitness_raw, fail_thr, w.bitmap, w.wcount, w.key,
                                           w.ctl);
    count_launch();
    FFG_TRY(check_launch("k_valid"));
    FFG_TRY(scan_exclusive(w.wcount, w.wprefix, W, w.scratch, stream));
    k_nodes<<<grid, kThreads, 0, stream>>>(R, w.key, w.bitmap, w.wprefix, w.node_of, w.nodes);
    count_launch();
    FFG_TRY(check_launch("k_nodes"));
    if (nbh == FFG_HAMMING)
        k_count<FFG_HAMMING><<<grid, kThreads, 0, stream>>>(d, w.nodes, w.key, w.outdeg,
                                                            w.indeg, w.ctl);
    else
        k_count<FFG_ADJACENT><<<grid, kThreads, 0, stream>>>(d, w.nodes, w.key, w.outdeg,
                                                             w.indeg, w.ctl);
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
    const int64_t N = g->n_nodes;
    const unsigned grid = static_cast<unsigned>((N + kThreads - 1) / kThreads);
    FFG_TRY(scan_exclusive(w.outdeg, g->out_ptr, N, w.scratch, stream));
    FFG_TRY(scan_exclusive(w.indeg, g->in_ptr, N, w.scratch, stream));
    if (nbh == FFG_HAMMING)
        k_emit<FFG_HAMMING><<<grid, kThreads, 0, stream>>>(
            d, N, w.nodes, w.key, w.node_of, g->out_ptr, g->in_ptr, g->out_idx,
            g->in_idx, g->outdeg, g->node_raw, g->is_min);
    else
        k_emit<FFG_ADJACENT><<<grid, kThreads, 0, stream>>>(
            d, N, w.nodes, w.key, w.node_of, g->out_ptr, g->in_ptr, g->out_idx,
            g->in_idx, g->outdeg, g->node_raw, g->is_min);
    count_launch();
    return check_launch("k_emit");
}

// ---------------------------------------------------------------------------
// batched construction: every job's count phase in four launches and one
// read-back, every fill in four launches.  Blocks map to jobs through a
// prefix of per-job block counts; per-job arrays are slices of arrays over
// all jobs, so each scan runs once over all jobs and a job's offsets are its
// slice minus the slice's first value.
// ---------------------------------------------------------------------------
namespace ffg {
namespace {

struct BJob {
    const DevSpace *sp;
    const double *fit;
    double fail_thr;
    int32_t nbh, pad;
    int64_t n_raw;
    int64_t woff, roff;  // first word / raw slot of the job in the arrays over all jobs
    // graph arrays (recorded by the fill) and the sizes the count reported
    int64_t *out_ptr, *in_ptr;
    int32_t *out_idx, *in_idx, *outdeg;
    int64_t *node_raw;
    uint8_t *is_min;
    int64_t n_nodes, n_edges;
};

struct BatchBuildWs {
    DevSpace *dsp;
    BJob *jobs;
    int64_t *blk0;    // n + 1: first block of every job
    int64_t *row0;    // n + 1: first row-pointer slot of every job (N + 1 per job)
    BuildCtl *ctl;    // n
    int32_t *status;  // n
    uint32_t *bitmap;
    int32_t *wcount;
    int64_t *wpre;
    int32_t *odeg, *ideg;
    int64_t *opre, *ipre;
    int64_t *scratch;
    unsigned long long *key;  // per raw point of every job (see key_of)
    int32_t *node_of;  // per raw point of every job
    int32_t *nodes;    // per node of every job (at the job's raw offset): its raw point
    int64_t *blk0n;    // n + 1: first node block of every job (from the device counts)
    size_t bytes;
};

BatchBuildWs carve_bb(void *base, int n, int64_t total_raw, int64_t total_words) {
    Carver c(base);
    BatchBuildWs w;
    w.dsp = c.take<DevSpace>(n);
    w.jobs = c.take<BJob>(n);
    w.blk0 = c.take<int64_t>(size_t(n) + 1);
    w.row0 = c.take<int64_t>(size_t(n) + 1);
    w.ctl = c.take<BuildCtl>(n);
    w.status = c.take<int32_t>(n);
    w.bitmap = c.take<uint32_t>(total_words);
    w.wcount = c.take<int32_t>(total_words);
    w.wpre = c.take<int64_t>(total_words + 1);
    w.odeg = c.take<int32_t>(total_raw);
    w.ideg = c.take<int32_t>(total_raw);
    w.opre = c.take<int64_t>(total_raw + 1);
    w.ipre = c.take<int64_t>(total_raw + 1);
    w.scratch = c.take<int64_t>(scan_scratch_elems(total_raw > total_words ? total_raw
                                                                           : total_words));
    w.key = c.take<unsigned long long>(total_raw);
    w.node_of = c.take<int32_t>(total_raw);
    w.nodes = c.take<int32_t>(total_raw);
    w.blk0n = c.take<int64_t>(size_t(n) + 1);
    w.bytes = c.off;
    return w;
}

// the job of a block (thread 0 searches, the block reads it from shared)
__device__ __forceinline__ int job_of_block(const int64_t *__restrict__ blk0, int n) {
    __shared__ int s_job;
    if (threadIdx.x == 0) {
        const int64_t b = blockIdx.x;
        int lo = 0, hi = n - 1;  // last job starting at or before b
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (blk0[mid] <= b) lo = mid;
            else hi = mid - 1;
        }
        s_job = lo;
    }
    __syncthreads();
    return s_job;
}

__global__ void k_bctl_init(BuildCtl *ctl, int32_t *status, int n) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        ctl[s].fopt_bits = ~0ULL;
        ctl[s].n_nodes = ctl[s].n_out = ctl[s].n_in = ctl[s].n_minima = 0;
        status[s] = 0;
    }
}

__global__ void __launch_bounds__(kThreads) k_valid_batch(const BJob *__restrict__ jobs,
                                                          const int64_t *__restrict__ blk0, int n,
                                                          uint32_t *bitmap, int32_t *wcount,
                                                          unsigned long long *key, BuildCtl *ctl) {
    __shared__ SmemSpace s;
    __shared__ int64_t vals[FFG_MAX_VALUES];
    const int j = job_of_block(blk0, n);
    const BJob &J = jobs[j];
    stage_space(*J.sp, s, vals, true);
    const int64_t r = (int64_t(blockIdx.x) - blk0[j]) * kThreads + threadIdx.x;
    valid_body(s, vals, J.n_raw, r, J.fit, J.fail_thr, bitmap + J.woff, wcount + J.woff,
               key + J.roff, ctl + j);
}

__global__ void __launch_bounds__(kThreads) k_nodes_batch(const BJob *__restrict__ jobs,
                                                          const int64_t *__restrict__ blk0, int n,
                                                          const unsigned long long *__restrict__ key,
                                                          const uint32_t *__restrict__ bitmap,
                                                          const int64_t *__restrict__ wpre,
                                                          int32_t *node_of, int32_t *nodes) {
    const int j = job_of_block(blk0, n);
    const BJob &J = jobs[j];
    const int64_t r = (int64_t(blockIdx.x) - blk0[j]) * kThreads + threadIdx.x;
    nodes_body(J.n_raw, r, key + J.roff, bitmap + J.woff, wpre + J.woff, wpre[J.woff],
               node_of + J.roff, nodes + J.roff);
}

// first node block of every job, from the node counts of the validity pass
__global__ void k_node_blocks(const BuildCtl *__restrict__ ctl, int n, int64_t *blk0n) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t b = 0;
    for (int j = 0; j < n; ++j) {
        blk0n[j] = b;
        b += (static_cast<int64_t>(ctl[j].n_nodes) + kThreads - 1) / kThreads;
    }
    blk0n[n] = b;
}

// one thread per node; blocks past the last job's nodes have nothing to do
__global__ void __launch_bounds__(kThreads) k_count_batch(const BJob *__restrict__ jobs,
                                                          const int64_t *__restrict__ blk0n, int n,
                                                          const unsigned long long *__restrict__ key,
                                                          const int32_t *__restrict__ nodes,
                                                          int32_t *odeg, int32_t *ideg,
                                                          BuildCtl *ctl) {
    if (int64_t(blockIdx.x) >= blk0n[n]) return;  // uniform over the block
    __shared__ SmemSpace s;
    const int j = job_of_block(blk0n, n);
    const BJob &J = jobs[j];
    stage_space(*J.sp, s, nullptr, false);
    const int64_t node = (int64_t(blockIdx.x) - blk0n[j]) * kThreads + threadIdx.x;
    const int64_t N = static_cast<int64_t>(ctl[j].n_nodes);
    if (J.nbh == FFG_HAMMING)
        count_body<FFG_HAMMING>(s, J.n_raw, N, node, nodes + J.roff, key + J.roff,
                                odeg + J.roff, ideg + J.roff, ctl + j);
    else
        count_body<FFG_ADJACENT>(s, J.n_raw, N, node, nodes + J.roff, key + J.roff,
                                 odeg + J.roff, ideg + J.roff, ctl + j);
}

// the device counts of job j equal the sizes its graph arrays were made for
__device__ __forceinline__ bool sizes_match(const BJob &J, const BuildCtl &c) {
    return static_cast<int64_t>(c.n_nodes) == J.n_nodes &&
           static_cast<int64_t>(c.n_out) == J.n_edges && c.n_in == c.n_out;
}

// out_ptr / in_ptr of every job: its slice of the scans, rebased
__global__ void k_rebase(const BJob *__restrict__ jobs, const int64_t *__restrict__ row0, int n,
                         int64_t total, const int64_t *__restrict__ opre,
                         const int64_t *__restrict__ ipre, const BuildCtl *__restrict__ ctl,
                         int32_t *status) {
    for (int64_t x = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; x < total;
         x += int64_t(gridDim.x) * blockDim.x) {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (row0[mid] <= x) lo = mid;
            else hi = mid - 1;
        }
        const BJob &J = jobs[lo];
        const int64_t i = x - row0[lo];
        if (!sizes_match(J, ctl[lo])) {
            if (i == 0) status[lo] = FFG_ERR_INVALID_ARG;
            continue;
        }
        J.out_ptr[i] = opre[J.roff + i] - opre[J.roff];
        J.in_ptr[i] = ipre[J.roff + i] - ipre[J.roff];
    }
}

__global__ void __launch_bounds__(kThreads) k_emit_batch(const BJob *__restrict__ jobs,
                                                         const int64_t *__restrict__ blk0n, int n,
                                                         const unsigned long long *__restrict__ key,
                                                         const int32_t *__restrict__ nodes,
                                                         const int32_t *__restrict__ node_of,
                                                         const BuildCtl *__restrict__ ctl) {
    if (int64_t(blockIdx.x) >= blk0n[n]) return;  // uniform over the block
    __shared__ SmemSpace s;
    const int j = job_of_block(blk0n, n);
    const BJob &J = jobs[j];
    if (!sizes_match(J, ctl[j])) return;  // uniform over the block
    stage_space(*J.sp, s, nullptr, false);
    const int64_t node = (int64_t(blockIdx.x) - blk0n[j]) * kThreads + threadIdx.x;
    if (J.nbh == FFG_HAMMING)
        emit_body<FFG_HAMMING>(s, J.n_raw, J.n_nodes, node, nodes + J.roff, key + J.roff,
                               node_of + J.roff, J.out_ptr, J.in_ptr, J.out_idx, J.in_idx,
                               J.outdeg, J.node_raw, J.is_min);
    else
        emit_body<FFG_ADJACENT>(s, J.n_raw, J.n_nodes, node, nodes + J.roff, key + J.roff,
                                node_of + J.roff, J.out_ptr, J.in_ptr, J.out_idx, J.in_idx,
                                J.outdeg, J.node_raw, J.is_min);
}

struct BatchSizes {
    int64_t total_raw = 0, total_words = 0, total_blocks = 0;
};

ffg_status batch_sizes(const ffg_build_job *jobs, int n, std::vector<DevSpace> *dsp,
                       BatchSizes *z) {
    if (!jobs || n < 1) return set_error("jobs NULL or n_jobs < 1"), FFG_ERR_INVALID_ARG;
    if (dsp) dsp->resize(n);
    DevSpace d;
    for (int j = 0; j < n; ++j) {
        const ffg_build_job &b = jobs[j];
        FFG_TRY(make_dev_space(b.space, dsp ? &(*dsp)[j] : &d));
        const DevSpace &x = dsp ? (*dsp)[j] : d;
        if (b.nbh != FFG_HAMMING && b.nbh != FFG_ADJACENT)
            return set_error("job %d: unknown neighbourhood %d", j, (int)b.nbh),
                   FFG_ERR_INVALID_ARG;
        if (!b.fitness_raw || !b.g || b.fail_thr != b.fail_thr)
            return set_error("job %d: fitness or graph NULL, or fail_thr NaN", j),
                   FFG_ERR_INVALID_ARG;
        z->total_raw += x.n_raw;
        z->total_words += (x.n_raw + 31) / 32;
        z->total_blocks += (x.n_raw + kThreads - 1) / kThreads;
    }
    if (z->total_blocks >= (int64_t(1) << 31))
        return set_error("too many raw points in one batch"), FFG_ERR_OVERFLOW;
    return FFG_OK;
}

unsigned grid_of(int64_t items, int threads) {
    const int64_t g = (items + threads - 1) / threads;
    return static_cast<unsigned>(g < 1 ? 1 : (g > 65535 * 32 ? 65535 * 32 : g));
}

// the count phase on the device (tables already in the workspace)
ffg_status launch_count_phase(const BatchBuildWs &w, int n, int64_t total_raw,
                              int64_t total_words, int64_t total_blocks, cudaStream_t stream) {
    k_bctl_init<<<grid_of(n, 128), 128, 0, stream>>>(w.ctl, w.status, n);
    count_launch();
    FFG_TRY(check_launch("k_bctl_init"));
    FFG_TRY(check_cuda(cudaMemsetAsync(w.odeg, 0, sizeof(int32_t) * total_raw, stream), "memset"));
    FFG_TRY(check_cuda(cudaMemsetAsync(w.ideg, 0, sizeof(int32_t) * total_raw, stream), "memset"));
    k_valid_batch<<<static_cast<unsigned>(total_blocks), kThreads, 0, stream>>>(
        w.jobs, w.blk0, n, w.bitmap, w.wcount, w.key, w.ctl);
    count_launch();
    FFG_TRY(check_launch("k_valid_batch"));
    FFG_TRY(scan_exclusive(w.wcount, w.wpre, total_words, w.scratch, stream));
    k_nodes_batch<<<static_cast<unsigned>(total_blocks), kThreads, 0, stream>>>(
        w.jobs, w.blk0, n, w.key, w.bitmap, w.wpre, w.node_of, w.nodes);
    count_launch();
    FFG_TRY(check_launch("k_nodes_batch"));
    k_node_blocks<<<1, 32, 0, stream>>>(w.ctl, n, w.blk0n);
    count_launch();
    FFG_TRY(check_launch("k_node_blocks"));
    // grid sized for every raw point: the node blocks are fewer
    k_count_batch<<<static_cast<unsigned>(total_blocks), kThreads, 0, stream>>>(
        w.jobs, w.blk0n, n, w.key, w.nodes, w.odeg, w.ideg, w.ctl);
    count_launch();
    return check_launch("k_count_batch");
}

// the fill phase on the device (graph pointers and sizes already recorded)
ffg_status launch_fill_phase(const BatchBuildWs &w, int n, int64_t total_raw, int64_t total_rows,
                             int64_t total_blocks, cudaStream_t stream) {
    FFG_TRY(scan_exclusive(w.odeg, w.opre, total_raw, w.scratch, stream));
    FFG_TRY(scan_exclusive(w.ideg, w.ipre, total_raw, w.scratch, stream));
    k_rebase<<<grid_of(total_rows, 256), 256, 0, stream>>>(w.jobs, w.row0, n, total_rows, w.opre,
                                                           w.ipre, w.ctl, w.status);
    count_launch();
    FFG_TRY(check_launch("k_rebase"));
    k_emit_batch<<<static_cast<unsigned>(total_blocks), kThreads, 0, stream>>>(
        w.jobs, w.blk0n, n, w.key, w.nodes, w.node_of, w.ctl);
    count_launch();
    return check_launch("k_emit_batch");
}

BatchBuildWs ws_of(const ffg_build_batch *plan) {
    BatchBuildWs w{};
    w.dsp = static_cast<DevSpace *>(plan->tables[0]);
    w.jobs = static_cast<BJob *>(plan->tables[1]);
    w.blk0 = static_cast<int64_t *>(plan->tables[2]);
    w.row0 = static_cast<int64_t *>(plan->tables[3]);
    w.ctl = static_cast<BuildCtl *>(plan->tables[4]);
    w.status = static_cast<int32_t *>(plan->tables[5]);
    w.bitmap = static_cast<uint32_t *>(plan->tables[6]);
    w.wcount = static_cast<int32_t *>(plan->tables[7]);
    w.wpre = static_cast<int64_t *>(plan->tables[8]);
    w.odeg = static_cast<int32_t *>(plan->tables[9]);
    w.ideg = static_cast<int32_t *>(plan->tables[10]);
    w.opre = static_cast<int64_t *>(plan->tables[11]);
    w.ipre = static_cast<int64_t *>(plan->tables[12]);
    w.scratch = static_cast<int64_t *>(plan->tables[13]);
    w.key = static_cast<unsigned long long *>(plan->tables[14]);
    w.node_of = static_cast<int32_t *>(plan->tables[15]);
    w.nodes = static_cast<int32_t *>(plan->tables[16]);
    w.blk0n = static_cast<int64_t *>(plan->tables[17]);
    return w;
}

}  // namespace
}  // namespace ffg

extern "C" size_t ffg_build_batch_workspace_bytes(const ffg_build_job *jobs, int32_t n_jobs) {
    clear_error();
    BatchSizes z;
    if (batch_sizes(jobs, n_jobs, nullptr, &z) != FFG_OK) return 0;
    return carve_bb(nullptr, n_jobs, z.total_raw, z.total_words).bytes;
}

extern "C" ffg_status ffg_build_batch_count(const ffg_build_job *jobs, int32_t n_jobs,
                                            void *workspace, size_t ws_bytes,
                                            ffg_build_batch *plan, void *stream_) {
    clear_error();
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    std::vector<DevSpace> dsp;
    BatchSizes z;
    FFG_TRY(batch_sizes(jobs, n_jobs, &dsp, &z));
    if (!plan || !workspace || !aligned256(workspace))
        return set_error("plan NULL or workspace NULL / not 256-byte aligned"),
               FFG_ERR_INVALID_ARG;
    BatchBuildWs w = carve_bb(workspace, n_jobs, z.total_raw, z.total_words);
    if (ws_bytes < w.bytes)
        return set_error("workspace %zu bytes, need %zu", ws_bytes, w.bytes), FFG_ERR_NO_MEMORY;
    std::vector<BJob> bj(n_jobs);
    std::vector<int64_t> blk0(n_jobs + 1, 0);
    int64_t woff = 0, roff = 0;
    for (int j = 0; j < n_jobs; ++j) {
        BJob &b = bj[j];
        b = BJob{};
        b.sp = w.dsp + j;
        b.fit = jobs[j].fitness_raw;
        b.fail_thr = jobs[j].fail_thr;
        b.nbh = jobs[j].nbh;
        b.n_raw = dsp[j].n_raw;
        b.woff = woff;
        b.roff = roff;
        b.n_nodes = b.n_edges = -1;  // no arrays yet: the fill kernels skip the job
        woff += (dsp[j].n_raw + 31) / 32;
        roff += dsp[j].n_raw;
        blk0[j + 1] = blk0[j] + (dsp[j].n_raw + kThreads - 1) / kThreads;
    }
    FFG_TRY(check_cuda(cudaMemcpyAsync(w.dsp, dsp.data(), sizeof(DevSpace) * n_jobs,
                                       cudaMemcpyHostToDevice, stream), "upload spaces"));
    FFG_TRY(check_cuda(cudaMemcpyAsync(w.jobs, bj.data(), sizeof(BJob) * n_jobs,
                                       cudaMemcpyHostToDevice, stream), "upload jobs"));
    FFG_TRY(check_cuda(cudaMemcpyAsync(w.blk0, blk0.data(), sizeof(int64_t) * (n_jobs + 1),
                                       cudaMemcpyHostToDevice, stream), "upload jobs"));
    FFG_TRY(launch_count_phase(w, n_jobs, z.total_raw, z.total_words, z.total_blocks, stream));
    std::vector<BuildCtl> h(n_jobs);
    FFG_TRY(check_cuda(cudaMemcpyAsync(h.data(), w.ctl, sizeof(BuildCtl) * n_jobs,
                                       cudaMemcpyDeviceToHost, stream), "read counts"));
    FFG_TRY(check_cuda(cudaStreamSynchronize(stream), "sync counts"));
    bool empty = false;
    for (int j = 0; j < n_jobs; ++j) {
        if (h[j].n_out != h[j].n_in) {
            set_error("internal: job %d out-degree sum != in-degree sum", j);
            return FFG_ERR_CUDA;
        }
        ffg_graph *g = jobs[j].g;
        g->n_raw = dsp[j].n_raw;
        g->n_nodes = static_cast<int64_t>(h[j].n_nodes);
        g->n_edges = static_cast<int64_t>(h[j].n_out);
        g->n_minima = static_cast<int64_t>(h[j].n_minima);
        g->f_opt = h[j].fopt_bits == ~0ULL ? __builtin_inf() : from_ordered_bits(h[j].fopt_bits);
        empty = empty || g->n_nodes == 0;
    }
    plan->n_jobs = n_jobs;
    plan->reserved = 0;
    plan->total_raw = z.total_raw;
    plan->total_words = z.total_words;
    plan->total_blocks = z.total_blocks;
    plan->total_rows = 0;
    void *t[] = {w.dsp,  w.jobs, w.blk0, w.row0, w.ctl,     w.status, w.bitmap,  w.wcount, w.wpre,
                 w.odeg, w.ideg, w.opre, w.ipre, w.scratch, w.key,    w.node_of, w.nodes,  w.blk0n};
    for (int k = 0; k < 18; ++k) plan->tables[k] = t[k];
    if (empty) return set_error("a job has no valid configuration"), FFG_ERR_EMPTY;
    return FFG_OK;
}

extern "C" ffg_status ffg_build_batch_fill(const ffg_build_job *jobs, int32_t n_jobs,
                                           ffg_build_batch *plan, void *stream_) {
    clear_error();
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (!jobs || !plan || n_jobs != plan->n_jobs || !plan->tables[1])
        return set_error("jobs do not match the plan of ffg_build_batch_count"),
               FFG_ERR_INVALID_ARG;
    BatchBuildWs w = ws_of(plan);
    std::vector<BJob> bj(n_jobs);
    FFG_TRY(check_cuda(cudaMemcpyAsync(bj.data(), w.jobs, sizeof(BJob) * n_jobs,
                                       cudaMemcpyDeviceToHost, stream), "read jobs"));
    FFG_TRY(check_cuda(cudaStreamSynchronize(stream), "sync jobs"));
    std::vector<int64_t> row0(n_jobs + 1, 0);
    for (int j = 0; j < n_jobs; ++j) {
        const ffg_graph *g = jobs[j].g;
        if (!g || g->n_raw != bj[j].n_raw || g->n_nodes <= 0 || g->n_nodes > g->n_raw ||
            g->n_edges < 0)
            return set_error("job %d: graph sizes do not come from ffg_build_batch_count", j),
                   FFG_ERR_INVALID_ARG;
        if (!g->out_ptr || !g->in_ptr || !g->outdeg || !g->node_raw || !g->is_min ||
            (g->n_edges > 0 && (!g->out_idx || !g->in_idx)))
            return set_error("job %d: a graph buffer is NULL", j), FFG_ERR_INVALID_ARG;
        BJob &b = bj[j];
        b.out_ptr = g->out_ptr;
        b.in_ptr = g->in_ptr;
        b.out_idx = g->out_idx;
        b.in_idx = g->in_idx;
        b.outdeg = g->outdeg;
        b.node_raw = g->node_raw;
        b.is_min = g->is_min;
        b.n_nodes = g->n_nodes;
        b.n_edges = g->n_edges;
        row0[j + 1] = row0[j] + g->n_nodes + 1;
    }
    FFG_TRY(check_cuda(cudaMemcpyAsync(w.jobs, bj.data(), sizeof(BJob) * n_jobs,
                                       cudaMemcpyHostToDevice, stream), "upload jobs"));
    FFG_TRY(check_cuda(cudaMemcpyAsync(w.row0, row0.data(), sizeof(int64_t) * (n_jobs + 1),
                                       cudaMemcpyHostToDevice, stream), "upload rows"));
    plan->total_rows = row0[n_jobs];
    FFG_TRY(launch_fill_phase(w, n_jobs, plan->total_raw, plan->total_rows, plan->total_blocks,
                              stream));
    // the host vectors die here: the copies above must have been read
    return check_cuda(cudaStreamSynchronize(stream), "sync fill upload");
}

extern "C" ffg_status ffg_build_batch_rerun(const ffg_build_batch *plan, void *stream_) {
    clear_error();
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (!plan || plan->n_jobs < 1 || !plan->tables[1] || plan->total_rows <= 0)
        return set_error("plan has not been filled"), FFG_ERR_INVALID_ARG;
    const BatchBuildWs w = ws_of(plan);
    FFG_TRY(launch_count_phase(w, plan->n_jobs, plan->total_raw, plan->total_words,
                               plan->total_blocks, stream));
    return launch_fill_phase(w, plan->n_jobs, plan->total_raw, plan->total_rows,
                             plan->total_blocks, stream);
}

extern "C" ffg_status ffg_build_batch_query(const ffg_build_batch *plan, int32_t *status_out,
                                            void *stream_) {
    clear_error();
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (!plan || plan->n_jobs < 1 || !plan->tables[5] || !status_out)
        return set_error("plan or status_out NULL"), FFG_ERR_INVALID_ARG;
    FFG_TRY(check_cuda(cudaMemcpyAsync(status_out, plan->tables[5], sizeof(int32_t) * plan->n_jobs,
                                       cudaMemcpyDeviceToHost, stream), "read status"));
    FFG_TRY(check_cuda(cudaStreamSynchronize(stream), "sync status"));
    ffg_status worst = FFG_OK;
    for (int j = 0; j < plan->n_jobs; ++j)
        if (status_out[j] != FFG_OK) worst = static_cast<ffg_status>(status_out[j]);
    if (worst != FFG_OK) set_error("a job's counts differ from the sizes of its arrays");
    return worst;
}

namespace ffg {
FFG_CHECK_READER(check_read_build)
}  // namespace ffg
