// ffg_pagerank.cu -- PageRank centrality on the FFG (Sec. VII-B), pull form.
//
// The matrix of Sec. VII-B is the adjacency matrix with every column scaled
// to sum to one, A[v,u] = 1/outdeg(u) for u -> v.  On an FFG (a DAG) A is
// nilpotent, so the damped form with uniform teleport and uniform
// redistribution of the mass of nodes without out-edges is used:
//   x'[v] = alpha * sum_{u in in(v)} w[u] + (alpha * D + 1 - alpha) / N,
//   w[u]  = x[u] / outdeg[u],   D = sum_{outdeg(u) = 0} x[u].
//
// One cooperative persistent launch runs every iteration.  Each block owns a
// contiguous range of rows, balanced by in-edges plus a per-row cost; rows
// are processed by groups of G lanes that stream the row's in_idx segment
// (4 loads in flight per lane) and gather w.  Only w is kept between
// iterations (ping-pong): x[v] = w[v] * outdeg[v] (or w[v] for a node
// without out-edges), so an iteration moves in_idx (4 B/edge), in_ptr and
// outdeg (12 B/row), the own w (read) and the new w (write).  Residual
// sum |x'-x|, next D and sum x' are reduced in FP64 per block, written to a
// double-buffered partials array, and after a grid barrier every block sums
// the partials in the same fixed order, so all blocks take the same
// stopping decision and the result is deterministic for a given grid.
// Barrier waits are bounded (globaltimer); on expiry the kernel records
// FFG_ERR_TIMEOUT and returns.
#include "ffg_internal.cuh"

namespace ffg {

namespace {

constexpr int kPrThreads = 256;
constexpr int kMaxBlocks = 4096;
constexpr int64_t kRowCost = 4;            // row cost in units of one in-edge
constexpr uint64_t kTimeoutNs = 2000000000ULL;

struct PrCtl {
    unsigned int barrier;
    int status;
    int iters;
    int converged;
    double residual;
    int nblocks;
    int pad;
};

struct PrWs {
    PrCtl *ctl;
    double *partials;  // [2][kMaxBlocks][4]
    void *w0, *w1;
    size_t bytes;
};

PrWs carve(void *base, int64_t n, size_t elem) {
    Carver c(base);
    PrWs w;
    w.ctl = c.take<PrCtl>(1);
    w.partials = c.take<double>(size_t(2) * kMaxBlocks * 4);
    w.w0 = c.take<char>(size_t(n) * elem);
    w.w1 = c.take<char>(size_t(n) * elem);
    w.bytes = c.off;
    return w;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier over a cooperative launch.  Bounded: gives up after
// kTimeoutNs (or 2^24 polls), records FFG_ERR_TIMEOUT.  Returns false
// (uniformly for the whole block) if the run must stop.
__device__ bool grid_barrier(PrCtl *ctl, unsigned target) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        red_release_add(&ctl->barrier, 1u);
        const uint64_t t0 = global_ns();
        unsigned ns = 32;
        int ok = 1;
        for (uint32_t polls = 0; ld_acquire(&ctl->barrier) < target; ++polls) {
            if (*(volatile int *)&ctl->status != 0) { ok = 0; break; }
            if (polls > (1u << 24) || global_ns() - t0 > kTimeoutNs) {
                atomicCAS(&ctl->status, 0, (int)FFG_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(ns);
            if (ns < 256) ns <<= 1;
        }
        __threadfence();
        if (*(volatile int *)&ctl->status != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block sums of three doubles; valid in thread 0
__device__ __forceinline__ void block_sum3(double &a, double &b, double &c) {
    __shared__ double red[3][kPrThreads / 32];
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        red[0][warp] = a;
        red[1][warp] = b;
        red[2][warp] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = b = c = 0.0;
        for (int k = 0; k < kPrThreads / 32; ++k) {
            a += red[0][k];
            b += red[1][k];
            c += red[2][k];
        }
    }
}

// every block sums the partials of all blocks in the same order (warp 0)
__device__ __forceinline__ void sum_partials(const double *part, int nb, double out[3]) {
    __shared__ double s_out[3];
    if (threadIdx.x < 32) {
        double a = 0, b = 0, c = 0;
        for (int k = threadIdx.x; k < nb; k += 32) {
            a += __ldcg(part + 4 * k + 0);
            b += __ldcg(part + 4 * k + 1);
            c += __ldcg(part + 4 * k + 2);
        }
        a = warp_sum(a);
        b = warp_sum(b);
        c = warp_sum(c);
        if (threadIdx.x == 0) {
            s_out[0] = a;
            s_out[1] = b;
            s_out[2] = c;
        }
    }
    __syncthreads();
    out[0] = s_out[0];
    out[1] = s_out[1];
    out[2] = s_out[2];
    __syncthreads();
}

__device__ __forceinline__ int64_t row_split(const int64_t *in_ptr, int64_t n, int b, int nb) {
    if (b <= 0) return 0;
    if (b >= nb) return n;
    const int64_t total = __ldg(in_ptr + n) + kRowCost * n;
    const int64_t target = total / nb * b + (total % nb) * b / nb;  // floor(total*b/nb)
    int64_t lo = 0, hi = n;  // smallest v with cost(v) >= target
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(in_ptr + mid) + kRowCost * mid >= target) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

template <typename T, int G>
__global__ void __launch_bounds__(kPrThreads) k_pagerank(
    const int64_t *__restrict__ in_ptr, const int32_t *__restrict__ in_idx,
    const int32_t *__restrict__ outdeg, int64_t n, double alpha, double tol, int max_iter,
    int init, T *ranks, T *w0, T *w1, double *partials, PrCtl *ctl) {
    const int nb = gridDim.x;
    __shared__ int64_t s_range[2];
    if (threadIdx.x == 0) {
        s_range[0] = row_split(in_ptr, n, blockIdx.x, nb);
        s_range[1] = row_split(in_ptr, n, blockIdx.x + 1, nb);
    }
    __syncthreads();
    const int64_t lo = s_range[0], hi = s_range[1];
    const int sub = threadIdx.x & (G - 1);
    const int group = threadIdx.x / G;
    constexpr int kGroups = kPrThreads / G;
    const double inv_n = 1.0 / static_cast<double>(n);

    // prologue: w from the start vector, D_0 and sum x_0
    {
        double dsum = 0.0, xsum = 0.0, unused = 0.0;
        for (int64_t v = lo + threadIdx.x; v < hi; v += kPrThreads) {
            const double x0 = init ? static_cast<double>(ranks[v]) : inv_n;
            const int32_t od = __ldg(outdeg + v);
            w0[v] = static_cast<T>(od ? x0 / od : x0);
            if (od == 0) dsum += x0;
            xsum += x0;
        }
        block_sum3(unused, dsum, xsum);
        if (threadIdx.x == 0) {
            double *p = partials + 4 * blockIdx.x;
            p[0] = 0.0;
            p[1] = dsum;
            p[2] = xsum;
        }
    }
    unsigned phase = 1;
    if (!grid_barrier(ctl, phase * nb)) return;
    double tot[3];
    sum_partials(partials, nb, tot);
    double dang = tot[1], xs = tot[2];
    double res = __longlong_as_double(0x7ff0000000000000LL), prev_res = res;
    int it = 0, converged = 0;
    T *wc = w0, *wn = w1;
    int par = 0;
    while (true) {
        const T c = static_cast<T>((alpha * dang + 1.0 - alpha) * inv_n);
        const T a = static_cast<T>(alpha);
        double r_acc = 0.0, d_acc = 0.0, s_acc = 0.0;
        for (int64_t base = lo; base < hi; base += kGroups) {
            const int64_t v = base + group;
            const bool active = v < hi;
            int64_t e = 0, end = 0;
            if (active) {
                e = __ldg(in_ptr + v) + sub;
                end = __ldg(in_ptr + v + 1);
            }
            T s = T(0);
            for (; e + 3 * G < end; e += 4 * G) {
                const int32_t i0 = __ldg(in_idx + e), i1 = __ldg(in_idx + e + G);
                const int32_t i2 = __ldg(in_idx + e + 2 * G), i3 = __ldg(in_idx + e + 3 * G);
                const T a0 = wc[i0], a1 = wc[i1], a2 = wc[i2], a3 = wc[i3];
                s += (a0 + a1) + (a2 + a3);
            }
            for (; e < end; e += G) s += wc[__ldg(in_idx + e)];
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (active && sub == 0) {
                const int32_t od = __ldg(outdeg + v);
                const T wv = wc[v];
                const T xo = od ? wv * static_cast<T>(od) : wv;
                const T xn = a * s + c;
                r_acc += fabs(static_cast<double>(xn) - static_cast<double>(xo));
                if (od == 0) d_acc += static_cast<double>(xn);
                s_acc += static_cast<double>(xn);
                wn[v] = od ? xn / static_cast<T>(od) : xn;
            }
        }
        block_sum3(r_acc, d_acc, s_acc);
        par ^= 1;
        double *pp = partials + size_t(par) * kMaxBlocks * 4;
        if (threadIdx.x == 0) {
            double *p = pp + 4 * blockIdx.x;
            p[0] = r_acc;
            p[1] = d_acc;
            p[2] = s_acc;
        }
        ++phase;
        if (!grid_barrier(ctl, phase * nb)) return;
        sum_partials(pp, nb, tot);
        prev_res = res;
        res = tot[0];
        dang = tot[1];
        xs = tot[2];
        ++it;
        T *t = wc;
        wc = wn;
        wn = t;
        if (res < tol) { converged = 1; break; }
        if (sizeof(T) == 4 && res >= prev_res) { converged = 1; break; }  // FP32 rounding floor
        if (it >= max_iter) break;
    }
    // epilogue: x' normalised to sum 1
    const double inv_s = 1.0 / xs;
    for (int64_t v = lo + threadIdx.x; v < hi; v += kPrThreads) {
        const int32_t od = __ldg(outdeg + v);
        const double x = od ? static_cast<double>(wc[v]) * od : static_cast<double>(wc[v]);
        ranks[v] = static_cast<T>(x * inv_s);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->iters = it;
        ctl->residual = res;
        ctl->converged = converged;
        ctl->nblocks = nb;
    }
}

template <typename T, int G>
ffg_status launch_g(const ffg_graph *g, double alpha, double tol, int max_iter, int init,
                    T *ranks, PrWs &w, cudaStream_t stream) {
    auto kern = k_pagerank<T, G>;
    int dev = 0, sms = 0, per_sm = 0;
    FFG_TRY(check_cuda(cudaGetDevice(&dev), "cudaGetDevice"));
    FFG_TRY(check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "attr"));
    FFG_TRY(check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPrThreads, 0),
                       "occupancy"));
    int64_t max_res = int64_t(sms) * per_sm;
    if (max_res > kMaxBlocks) max_res = kMaxBlocks;
    // at least ~8 row batches per block
    const int64_t rows_per_block = int64_t(kPrThreads / G) * 8;
    int64_t want = (g->n_nodes + rows_per_block - 1) / rows_per_block;
    int nb = static_cast<int>(want < 1 ? 1 : (want > max_res ? max_res : want));
    if (nb < 1) return set_error("kernel does not fit on the device"), FFG_ERR_CUDA;
    const int64_t *in_ptr = g->in_ptr;
    const int32_t *in_idx = g->in_idx;
    const int32_t *outdeg = g->outdeg;
    int64_t n = g->n_nodes;
    T *w0 = static_cast<T *>(w.w0), *w1 = static_cast<T *>(w.w1);
    double *partials = w.partials;
    PrCtl *ctl = w.ctl;
    void *args[] = {(void *)&in_ptr, (void *)&in_idx, (void *)&outdeg, (void *)&n,
                    (void *)&alpha, (void *)&tol, (void *)&max_iter, (void *)&init,
                    (void *)&ranks, (void *)&w0, (void *)&w1, (void *)&partials,
                    (void *)&ctl};
    FFG_TRY(check_cuda(cudaLaunchCooperativeKernel((const void *)kern, dim3(nb), dim3(kPrThreads),
                                                   args, 0, stream),
                       "k_pagerank"));
    count_launch();
    return FFG_OK;
}

template <typename T>
ffg_status launch(const ffg_graph *g, double alpha, double tol, int max_iter, int init,
                  T *ranks, PrWs &w, cudaStream_t stream) {
    const double avg = g->n_nodes ? double(g->n_edges) / double(g->n_nodes) : 0.0;
    if (avg >= 48) return launch_g<T, 16>(g, alpha, tol, max_iter, init, ranks, w, stream);
    if (avg >= 20) return launch_g<T, 8>(g, alpha, tol, max_iter, init, ranks, w, stream);
    if (avg >= 6) return launch_g<T, 4>(g, alpha, tol, max_iter, init, ranks, w, stream);
    return launch_g<T, 2>(g, alpha, tol, max_iter, init, ranks, w, stream);
}

ffg_status read_result(const PrCtl *dctl, int32_t *iters_out, double *residual_out,
                       cudaStream_t stream) {
    PrCtl h;
    FFG_TRY(check_cuda(cudaMemcpyAsync(&h, dctl, sizeof(h), cudaMemcpyDeviceToHost, stream),
                       "read pagerank result"));
    FFG_TRY(check_cuda(cudaStreamSynchronize(stream), "sync pagerank"));
    if (iters_out) *iters_out = h.iters;
    if (residual_out) *residual_out = h.residual;
    if (h.status != 0) {
        set_error("pagerank: device barrier timed out");
        return static_cast<ffg_status>(h.status);
    }
    return h.converged ? FFG_OK : FFG_ERR_NOT_CONVERGED;
}

}  // namespace

}  // namespace ffg

using namespace ffg;

extern "C" size_t pagerank_workspace_bytes(int64_t n_nodes, ffg_prec prec) {
    if (n_nodes < 0) return 0;
    return carve(nullptr, n_nodes, prec == FFG_F32 ? 4 : 8).bytes;
}

extern "C" ffg_status pagerank_solve(const ffg_graph *g, double damping, double tol,
                                     int32_t max_iter, ffg_prec prec, void *ranks, int init,
                                     void *workspace, size_t ws_bytes, int32_t *iters_out,
                                     double *residual_out, void *stream_) {
    clear_error();
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (!g || g->n_nodes <= 0 || !g->in_ptr || !g->outdeg || (g->n_edges > 0 && !g->in_idx))
        return set_error("graph is empty or incomplete"), FFG_ERR_INVALID_ARG;
    if (g->n_nodes >= (int64_t(1) << 31)) return set_error("too many nodes"), FFG_ERR_OVERFLOW;
    if (!(damping > 0.0 && damping < 1.0))
        return set_error("damping must lie in (0,1)"), FFG_ERR_INVALID_ARG;
    if (!(tol >= 0.0) || max_iter < 1)
        return set_error("tol must be >= 0 and max_iter >= 1"), FFG_ERR_INVALID_ARG;
    if (prec != FFG_F64 && prec != FFG_F32)
        return set_error("unknown precision %d", (int)prec), FFG_ERR_INVALID_ARG;
    if (!ranks || !workspace) return set_error("ranks/workspace NULL"), FFG_ERR_INVALID_ARG;
    if (!aligned256(workspace))
        return set_error("workspace not 256-byte aligned"), FFG_ERR_INVALID_ARG;
    PrWs w = carve(workspace, g->n_nodes, prec == FFG_F32 ? 4 : 8);
    if (ws_bytes < w.bytes)
        return set_error("workspace %zu bytes, need %zu", ws_bytes, w.bytes), FFG_ERR_NO_MEMORY;
    FFG_TRY(check_cuda(cudaMemsetAsync(w.ctl, 0, sizeof(PrCtl), stream), "memset"));
    if (prec == FFG_F64)
        FFG_TRY(launch<double>(g, damping, tol, max_iter, init, static_cast<double *>(ranks), w,
                               stream));
    else
        FFG_TRY(launch<float>(g, damping, tol, max_iter, init, static_cast<float *>(ranks), w,
                              stream));
    if (!iters_out && !residual_out) return FFG_OK;
    return read_result(w.ctl, iters_out, residual_out, stream);
}

extern "C" ffg_status pagerank_query(const void *workspace, int32_t *iters_out,
                                     double *residual_out, void *stream_) {
    clear_error();
    if (!workspace || !aligned256(workspace))
        return set_error("workspace NULL or misaligned"), FFG_ERR_INVALID_ARG;
    const PrCtl *ctl = static_cast<const PrCtl *>(workspace);
    return read_result(ctl, iters_out, residual_out, static_cast<cudaStream_t>(stream_));
}
