// ffg_centrality.cu -- p-proportion of centrality C_p (Sec. VII-B, Eq. 3).
//
// C_p = sum_{v in L_p} x[v] / sum_{v in L} x[v], L = local minima, L_p = the
// minima with f(v) <= (1 + p) f_opt.  With the thresholds sorted ascending,
// a minimum with fitness f falls in bucket b = the first threshold k with
// f <= thr_k (b = n_p if none); S_p(k) is then the sum of buckets 0..k and
// S_L the sum of all buckets.  One pass over the nodes fills per-block
// bucket sums (FP64: per thread, then a warp tree, then compensated across
// warps), a second one-block launch adds the blocks' buckets in a fixed
// order with Neumaier's compensated sum, and the host forms the prefix sums
// and the ratios in FP64.  The threshold decision f <= thr_k is taken in FP64
// with thr_k computed on the host as f_opt * (1 + p_k).
#include <algorithm>
#include <numeric>
#include <vector>

#include "ffg_internal.cuh"

namespace ffg {

namespace {

constexpr int kCpThreads = 256;
constexpr int kMaxCpBlocks = 1024;
constexpr int kBuckets = FFG_MAX_P + 1;

struct Thresholds {
    double thr[FFG_MAX_P];
    int n;
};

struct CpWs {
    double *partials;  // [kMaxCpBlocks][kBuckets][2] (sum, compensation)
    double *buckets;   // [kBuckets]
    size_t bytes;
};

CpWs carve(void *base) {
    Carver c(base);
    CpWs w;
    w.partials = c.take<double>(size_t(kMaxCpBlocks) * kBuckets * 2);
    w.buckets = c.take<double>(kBuckets);
    w.bytes = c.off;
    return w;
}

__device__ __forceinline__ void neumaier(double &s, double &c, double v) {
    const double t = s + v;
    if (fabs(s) >= fabs(v)) c += (s - t) + v;
    else c += (v - t) + s;
    s = t;
}

template <typename T>
__global__ void __launch_bounds__(kCpThreads) k_cp_partial(
    int64_t n, int64_t n_raw, const uint8_t *__restrict__ is_min,
    const int64_t *__restrict__ node_raw,
    const double *__restrict__ fit, const T *__restrict__ x, const Thresholds th,
    double *__restrict__ partials) {
    double acc[kBuckets];
    for (int b = 0; b <= th.n; ++b) acc[b] = 0.0;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (!is_min[v]) continue;
        const int64_t rv = node_raw[v];
        if (!FFG_CHECK(rv >= 0 && rv < n_raw, 501)) continue;
        const double f = fit[rv];
        int b = 0;
        while (b < th.n && !(f <= th.thr[b])) ++b;
        acc[b] += static_cast<double>(x[v]);
    }
    __shared__ double red[kCpThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int b = 0; b <= th.n; ++b) {
        double v = acc[b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        __syncthreads();
        if (lane == 0) red[warp] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0, c = 0.0;
            for (int k = 0; k < kCpThreads / 32; ++k) neumaier(s, c, red[k]);
            partials[(size_t(blockIdx.x) * kBuckets + b) * 2 + 0] = s;
            partials[(size_t(blockIdx.x) * kBuckets + b) * 2 + 1] = c;
        }
    }
}

// one warp per bucket: lanes add strided blocks with Neumaier's sum, then the
// 32 (sum, compensation) pairs are combined by lane 0 in lane order
__global__ void k_cp_final(const double *__restrict__ partials, int nblocks, int nb,
                           double *__restrict__ buckets) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    __shared__ double red[32][32][2];
    for (int b = warp; b <= nb; b += nwarps) {
        double s = 0.0, c = 0.0;
        for (int k = lane; k < nblocks; k += 32) {
            neumaier(s, c, partials[(size_t(k) * kBuckets + b) * 2 + 0]);
            neumaier(s, c, partials[(size_t(k) * kBuckets + b) * 2 + 1]);
        }
        red[warp][lane][0] = s;
        red[warp][lane][1] = c;
        __syncwarp();
        if (lane == 0) {
            double ts = 0.0, tc = 0.0;
            for (int k = 0; k < 32; ++k) {
                neumaier(ts, tc, red[warp][k][0]);
                neumaier(ts, tc, red[warp][k][1]);
            }
            buckets[b] = ts + tc;
        }
        __syncwarp();
    }
}

// the same compensated sum on the device (same operations, same order)
__device__ double dev_neumaier(const double *v, int n) {
    double s = 0.0, c = 0.0;
    for (int k = 0; k < n; ++k) neumaier(s, c, v[k]);
    return s + c;
}

double host_neumaier(const double *v, int n) {
    double s = 0.0, c = 0.0;
    for (int k = 0; k < n; ++k) {
        const double t = s + v[k];
        if (std::fabs(s) >= std::fabs(v[k])) c += (s - t) + v[k];
        else c += (v[k] - t) + s;
        s = t;
    }
    return s + c;
}

}  // namespace

}  // namespace ffg

using namespace ffg;

extern "C" size_t centrality_workspace_bytes(int32_t n_p) {
    (void)n_p;
    return carve(nullptr).bytes;
}

extern "C" ffg_status centrality_proportion(const ffg_graph *g, const double *fitness_raw,
                                            const void *ranks, ffg_prec prec, const double *p,
                                            int32_t n_p, double *cp_out, void *workspace,
                                            size_t ws_bytes, void *stream_) {
    clear_error();
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (!g || g->n_nodes <= 0 || !g->is_min || !g->node_raw)
        return set_error("graph is empty or incomplete"), FFG_ERR_INVALID_ARG;
    if (!fitness_raw || !ranks || !p || !cp_out || !workspace)
        return set_error("a pointer argument is NULL"), FFG_ERR_INVALID_ARG;
    if (n_p < 1 || n_p > FFG_MAX_P)
        return set_error("n_p must lie in [1,%d]", FFG_MAX_P), FFG_ERR_INVALID_ARG;
    if (prec != FFG_F64 && prec != FFG_F32)
        return set_error("unknown precision"), FFG_ERR_INVALID_ARG;
    for (int k = 0; k < n_p; ++k)
        if (!(p[k] >= 0.0) || p[k] == __builtin_inf())
            return set_error("p[%d] must be finite and >= 0", k), FFG_ERR_INVALID_ARG;
    if (!aligned256(workspace))
        return set_error("workspace not 256-byte aligned"), FFG_ERR_INVALID_ARG;
    CpWs w = carve(workspace);
    if (ws_bytes < w.bytes)
        return set_error("workspace %zu bytes, need %zu", ws_bytes, w.bytes), FFG_ERR_NO_MEMORY;
    if (g->n_minima <= 0) return set_error("the graph has no local minimum"), FFG_ERR_EMPTY;

    // thresholds in FP64 on the host: (1 + p) first, then the product
    std::vector<int> order(n_p);
    std::vector<double> thr(n_p);
    for (int k = 0; k < n_p; ++k) {
        volatile double onep = 1.0 + p[k];
        thr[k] = g->f_opt * onep;
    }
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return thr[a] < thr[b]; });
    Thresholds th;
    th.n = n_p;
    for (int k = 0; k < n_p; ++k) th.thr[k] = thr[order[k]];

    int dev = 0, sms = 0;
    FFG_TRY(check_cuda(cudaGetDevice(&dev), "cudaGetDevice"));
    FFG_TRY(check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "attr"));
    int64_t want = (g->n_nodes + kCpThreads - 1) / kCpThreads;
    int nblocks = static_cast<int>(std::min<int64_t>(want, std::min(kMaxCpBlocks, sms * 4)));
    if (nblocks < 1) nblocks = 1;
    if (prec == FFG_F64)
        k_cp_partial<double><<<nblocks, kCpThreads, 0, stream>>>(
            g->n_nodes, g->n_raw, g->is_min, g->node_raw, fitness_raw,
            static_cast<const double *>(ranks), th, w.partials);
    else
        k_cp_partial<float><<<nblocks, kCpThreads, 0, stream>>>(
            g->n_nodes, g->n_raw, g->is_min, g->node_raw, fitness_raw,
            static_cast<const float *>(ranks), th, w.partials);
    FFG_TRY(check_launch("k_cp_partial"));
    k_cp_final<<<1, 32 * std::min(n_p + 1, 32), 0, stream>>>(w.partials, nblocks, n_p, w.buckets);
    count_launch(2);
    FFG_TRY(check_launch("k_cp_final"));
    double h[kBuckets];
    FFG_TRY(check_cuda(cudaMemcpyAsync(h, w.buckets, sizeof(double) * (n_p + 1),
                                       cudaMemcpyDeviceToHost, stream),
                       "read buckets"));
    FFG_TRY(check_cuda(cudaStreamSynchronize(stream), "sync centrality"));
    const double sl = host_neumaier(h, n_p + 1);
    if (!(sl > 0.0)) return set_error("minima hold no centrality"), FFG_ERR_EMPTY;
    for (int k = 0; k < n_p; ++k) cp_out[order[k]] = host_neumaier(h, k + 1) / sl;
    return FFG_OK;
}

// ---------------------------------------------------------------------------
// batched C_p, planned once and re-run with launches only (capturable in a
// CUDA graph).  f_opt is taken on the device as the smallest fitness of a
// local minimum -- the global optimum is a local minimum (no neighbour is
// better) and no minimum is failed, so this is the build's f_opt -- and the
// thresholds f_opt * (1 + p_k) are formed there with the same two roundings
// as on the host.  Per run: a reset of the per-job minima, one launch for
// the minima (blockIdx.y = job), one for the bucket sums of every job, one
// for the per-job final sums and ratios (written to device memory).
// ---------------------------------------------------------------------------
namespace ffg {
namespace {

constexpr int kCpBatchBlocks = 32;

struct CpJobDev {
    const uint8_t *is_min;
    const int64_t *node_raw;
    const double *fit;
    const void *ranks;
    int64_t n, n_raw;
};

struct CpBatchWs {
    CpJobDev *jobs;
    double *p;                    // n_p fractions
    unsigned long long *fopt;     // per job: ordered bits of the smallest minimum fitness
    double *partials;
    double *buckets;
    double *cp;                   // n_jobs x n_p
    int32_t *status;              // per job
    size_t bytes;
};

CpBatchWs carve_cp_batch(void *base, int n_jobs) {
    Carver c(base);
    CpBatchWs w;
    w.jobs = c.take<CpJobDev>(n_jobs);
    w.p = c.take<double>(FFG_MAX_P);
    w.fopt = c.take<unsigned long long>(n_jobs);
    w.partials = c.take<double>(size_t(n_jobs) * kCpBatchBlocks * kBuckets * 2);
    w.buckets = c.take<double>(size_t(n_jobs) * kBuckets);
    w.cp = c.take<double>(size_t(n_jobs) * FFG_MAX_P);
    w.status = c.take<int32_t>(n_jobs);
    w.bytes = c.off;
    return w;
}

// smallest fitness over the job's local minima (ordered bits, atomicMin)
__global__ void __launch_bounds__(kCpThreads) k_cp_fopt_batch(const CpJobDev *__restrict__ jobs,
                                                               unsigned long long *fopt) {
    const CpJobDev &J = jobs[blockIdx.y];
    unsigned long long m = ~0ULL;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < J.n; v += stride)
        if (J.is_min[v] && FFG_CHECK(J.node_raw[v] >= 0 && J.node_raw[v] < J.n_raw, 501)) {
            const unsigned long long b = ordered_bits(J.fit[J.node_raw[v]]);
            m = b < m ? b : m;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
        m = t < m ? t : m;
    }
    if ((threadIdx.x & 31) == 0 && m != ~0ULL) atomicMin(fopt + blockIdx.y, m);
}

// the job's thresholds in ascending order and the position of each p:
// thr_k = f_opt * (1 + p_k), (1 + p_k) rounded first; equal thresholds keep
// the order of p (a stable sort, as on the host)
__device__ void cp_thresholds(unsigned long long fbits, const double *__restrict__ p, int n_p,
                              Thresholds &th, int *order) {
    const double f_opt = fbits == ~0ULL ? __builtin_nan("") : from_ordered_bits(fbits);
    double thr[FFG_MAX_P];
    for (int k = 0; k < n_p; ++k) thr[k] = __dmul_rn(f_opt, __dadd_rn(1.0, p[k]));
    for (int k = 0; k < n_p; ++k) order[k] = k;
    for (int i = 1; i < n_p; ++i) {  // insertion sort: stable
        const int o = order[i];
        int j = i - 1;
        while (j >= 0 && thr[order[j]] > thr[o]) {
            order[j + 1] = order[j];
            --j;
        }
        order[j + 1] = o;
    }
    th.n = n_p;
    for (int k = 0; k < n_p; ++k) th.thr[k] = thr[order[k]];
}

template <typename T>
__global__ void __launch_bounds__(kCpThreads) k_cp_partial_batch(
    const CpJobDev *__restrict__ jobs, const double *__restrict__ p, int n_p,
    const unsigned long long *__restrict__ fopt, double *__restrict__ partials) {
    const CpJobDev &J = jobs[blockIdx.y];
    __shared__ Thresholds s_th;
    if (threadIdx.x == 0) {
        int order[FFG_MAX_P];
        cp_thresholds(fopt[blockIdx.y], p, n_p, s_th, order);
    }
    __syncthreads();
    const T *x = static_cast<const T *>(J.ranks);
    double acc[kBuckets];
    for (int b = 0; b <= n_p; ++b) acc[b] = 0.0;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < J.n; v += stride) {
        if (!J.is_min[v]) continue;
        if (!FFG_CHECK(J.node_raw[v] >= 0 && J.node_raw[v] < J.n_raw, 501)) continue;
        const double f = J.fit[J.node_raw[v]];
        int b = 0;
        while (b < n_p && !(f <= s_th.thr[b])) ++b;
        acc[b] += static_cast<double>(x[v]);
    }
    __shared__ double red[kCpThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double *out = partials + (size_t(blockIdx.y) * kCpBatchBlocks + blockIdx.x) * kBuckets * 2;
    for (int b = 0; b <= n_p; ++b) {
        double v = acc[b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        __syncthreads();
        if (lane == 0) red[warp] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0, c = 0.0;
            for (int k = 0; k < kCpThreads / 32; ++k) neumaier(s, c, red[k]);
            out[b * 2 + 0] = s;
            out[b * 2 + 1] = c;
        }
    }
}

// block j: lane-strided compensated sums of job j's block partials per
// bucket, then C_p of every p (compensated prefix sums over the sum over
// all buckets), or NaN and FFG_ERR_EMPTY when the minima hold nothing
__global__ void k_cp_final_batch(const double *__restrict__ partials, const double *__restrict__ p,
                                 int n_p, const unsigned long long *__restrict__ fopt,
                                 double *__restrict__ buckets, double *__restrict__ cp,
                                 int32_t *__restrict__ status) {
    const int job = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    __shared__ double red[32][32][2];
    const double *base = partials + size_t(job) * kCpBatchBlocks * kBuckets * 2;
    double *bk = buckets + size_t(job) * kBuckets;
    for (int b = warp; b <= n_p; b += nwarps) {
        double s = 0.0, c = 0.0;
        for (int k = lane; k < kCpBatchBlocks; k += 32) {
            neumaier(s, c, base[(size_t(k) * kBuckets + b) * 2 + 0]);
            neumaier(s, c, base[(size_t(k) * kBuckets + b) * 2 + 1]);
        }
        red[warp][lane][0] = s;
        red[warp][lane][1] = c;
        __syncwarp();
        if (lane == 0) {
            double ts = 0.0, tc = 0.0;
            for (int k = 0; k < 32; ++k) {
                neumaier(ts, tc, red[warp][k][0]);
                neumaier(ts, tc, red[warp][k][1]);
            }
            bk[b] = ts + tc;
        }
        __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Thresholds th;
        int order[FFG_MAX_P];
        cp_thresholds(fopt[job], p, n_p, th, order);
        const double sl = dev_neumaier(bk, n_p + 1);
        const bool ok = sl > 0.0;
        for (int k = 0; k < n_p; ++k)
            cp[size_t(job) * n_p + order[k]] = ok ? dev_neumaier(bk, k + 1) / sl
                                                  : __builtin_nan("");
        status[job] = ok ? FFG_OK : FFG_ERR_EMPTY;
    }
}

ffg_status cp_batch_check(const ffg_cp_batch *plan) {
    if (!plan || plan->n_jobs < 1 || plan->n_jobs > 65535 || plan->n_p < 1 ||
        plan->n_p > FFG_MAX_P || !plan->tables[0] || !plan->cp || !plan->status ||
        (plan->prec != FFG_F64 && plan->prec != FFG_F32))
        return set_error("C_p plan is empty or incomplete"), FFG_ERR_INVALID_ARG;
    return FFG_OK;
}

}  // namespace
}  // namespace ffg

extern "C" size_t centrality_batch_workspace_bytes(int32_t n_jobs, int32_t n_p) {
    (void)n_p;
    if (n_jobs < 1 || n_jobs > 65535) return 0;
    return carve_cp_batch(nullptr, n_jobs).bytes;
}

extern "C" ffg_status centrality_batch_plan(const ffg_cp_job *jobs, int32_t n_jobs,
                                            ffg_prec prec, const double *p, int32_t n_p,
                                            void *workspace, size_t ws_bytes,
                                            ffg_cp_batch *plan, void *stream_) {
    clear_error();
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (!jobs || n_jobs < 1 || n_jobs > 65535 || !p || !plan || !workspace)
        return set_error("jobs, p, plan, workspace non-NULL and 1 <= n_jobs <= 65535"),
               FFG_ERR_INVALID_ARG;
    if (n_p < 1 || n_p > FFG_MAX_P)
        return set_error("n_p must lie in [1,%d]", FFG_MAX_P), FFG_ERR_INVALID_ARG;
    if (prec != FFG_F64 && prec != FFG_F32)
        return set_error("unknown precision"), FFG_ERR_INVALID_ARG;
    for (int k = 0; k < n_p; ++k)
        if (!(p[k] >= 0.0) || p[k] == __builtin_inf())
            return set_error("p[%d] must be finite and >= 0", k), FFG_ERR_INVALID_ARG;
    if (!aligned256(workspace))
        return set_error("workspace not 256-byte aligned"), FFG_ERR_INVALID_ARG;
    CpBatchWs w = carve_cp_batch(workspace, n_jobs);
    if (ws_bytes < w.bytes)
        return set_error("workspace %zu bytes, need %zu", ws_bytes, w.bytes), FFG_ERR_NO_MEMORY;
    std::vector<CpJobDev> jd(n_jobs);
    for (int j = 0; j < n_jobs; ++j) {
        const ffg_graph *g = jobs[j].g;
        if (!g || g->n_nodes <= 0 || !g->is_min || !g->node_raw || !jobs[j].fitness_raw ||
            !jobs[j].ranks)
            return set_error("job %d: graph, fitness or ranks missing", j), FFG_ERR_INVALID_ARG;
        jd[j].is_min = g->is_min;
        jd[j].node_raw = g->node_raw;
        jd[j].fit = jobs[j].fitness_raw;
        jd[j].ranks = jobs[j].ranks;
        jd[j].n = g->n_nodes;
        jd[j].n_raw = g->n_raw;
    }
    FFG_TRY(check_cuda(cudaMemcpyAsync(w.jobs, jd.data(), sizeof(CpJobDev) * n_jobs,
                                       cudaMemcpyHostToDevice, stream), "upload jobs"));
    FFG_TRY(check_cuda(cudaMemcpyAsync(w.p, p, sizeof(double) * n_p, cudaMemcpyHostToDevice,
                                       stream), "upload p"));
    FFG_TRY(check_cuda(cudaStreamSynchronize(stream), "sync C_p plan"));
    plan->n_jobs = n_jobs;
    plan->n_p = n_p;
    plan->prec = prec;
    plan->reserved = 0;
    plan->cp = w.cp;
    plan->status = w.status;
    plan->tables[0] = w.jobs;
    plan->tables[1] = w.p;
    plan->tables[2] = w.fopt;
    plan->tables[3] = w.partials;
    plan->tables[4] = w.buckets;
    return FFG_OK;
}

extern "C" ffg_status centrality_batch_run(const ffg_cp_batch *plan, void *stream_) {
    clear_error();
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    FFG_TRY(cp_batch_check(plan));
    const CpJobDev *jobs = static_cast<const CpJobDev *>(plan->tables[0]);
    const double *p = static_cast<const double *>(plan->tables[1]);
    unsigned long long *fopt = static_cast<unsigned long long *>(plan->tables[2]);
    double *partials = static_cast<double *>(plan->tables[3]);
    double *buckets = static_cast<double *>(plan->tables[4]);
    const int n_jobs = plan->n_jobs, n_p = plan->n_p;
    FFG_TRY(check_cuda(cudaMemsetAsync(fopt, 0xff, sizeof(unsigned long long) * n_jobs, stream),
                       "memset"));
    const dim3 grid(kCpBatchBlocks, n_jobs);
    k_cp_fopt_batch<<<grid, kCpThreads, 0, stream>>>(jobs, fopt);
    FFG_TRY(check_launch("k_cp_fopt_batch"));
    if (plan->prec == FFG_F64)
        k_cp_partial_batch<double><<<grid, kCpThreads, 0, stream>>>(jobs, p, n_p, fopt, partials);
    else
        k_cp_partial_batch<float><<<grid, kCpThreads, 0, stream>>>(jobs, p, n_p, fopt, partials);
    FFG_TRY(check_launch("k_cp_partial_batch"));
    k_cp_final_batch<<<n_jobs, 32 * std::min(n_p + 1, 32), 0, stream>>>(
        partials, p, n_p, fopt, buckets, plan->cp, plan->status);
    count_launch(3);
    return check_launch("k_cp_final_batch");
}

extern "C" ffg_status centrality_batch_query(const ffg_cp_batch *plan, double *cp_out,
                                             int32_t *status_out, void *stream_) {
    clear_error();
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    FFG_TRY(cp_batch_check(plan));
    std::vector<int32_t> st(plan->n_jobs);
    if (cp_out)
        FFG_TRY(check_cuda(cudaMemcpyAsync(cp_out, plan->cp,
                                           sizeof(double) * plan->n_jobs * plan->n_p,
                                           cudaMemcpyDeviceToHost, stream), "read C_p"));
    FFG_TRY(check_cuda(cudaMemcpyAsync(st.data(), plan->status, sizeof(int32_t) * st.size(),
                                       cudaMemcpyDeviceToHost, stream), "read C_p status"));
    FFG_TRY(check_cuda(cudaStreamSynchronize(stream), "sync C_p"));
    if (status_out) std::copy(st.begin(), st.end(), status_out);
    for (int32_t s : st)
        if (s != FFG_OK)
            return set_error("a job's graph has no local minimum (its C_p is NaN)"), FFG_ERR_EMPTY;
    return FFG_OK;
}

extern "C" ffg_status centrality_batch(const ffg_cp_job *jobs, int32_t n_jobs, ffg_prec prec,
                                       const double *p, int32_t n_p, double *cp_out,
                                       void *workspace, size_t ws_bytes, void *stream) {
    if (!cp_out) {
        clear_error();
        return set_error("cp_out is NULL"), FFG_ERR_INVALID_ARG;
    }
    ffg_cp_batch plan;
    FFG_TRY(centrality_batch_plan(jobs, n_jobs, prec, p, n_p, workspace, ws_bytes, &plan, stream));
    FFG_TRY(centrality_batch_run(&plan, stream));
    return centrality_batch_query(&plan, cp_out, nullptr, stream);
}

// ---------------------------------------------------------------------------
// the naive metric (Sec. VII-A): fraction of optimal fitness f_opt / f(x) of
// every local minimum, in ascending node order (flags, one scan, scatter)
// ---------------------------------------------------------------------------
namespace ffg {
namespace {

__global__ void k_min_flags(const uint8_t *__restrict__ is_min, int64_t n, int32_t *flag) {
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
         v += int64_t(gridDim.x) * blockDim.x)
        flag[v] = is_min[v] ? 1 : 0;
}

__global__ void k_min_emit(const uint8_t *__restrict__ is_min,
                           const int64_t *__restrict__ node_raw,
                           const double *__restrict__ fit, const int64_t *__restrict__ pos,
                           int64_t n, int64_t n_raw, double f_opt, double *frac, int64_t *node) {
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
         v += int64_t(gridDim.x) * blockDim.x) {
        if (!is_min[v]) continue;
        const int64_t k = pos[v];
        if (!FFG_CHECK(node_raw[v] >= 0 && node_raw[v] < n_raw, 502)) continue;
        frac[k] = f_opt / fit[node_raw[v]];
        if (node) node[k] = v;
    }
}

unsigned min_grid(int64_t n) {
    const int64_t g = (n + 255) / 256;
    return static_cast<unsigned>(g < 1 ? 1 : (g > 65535 ? 65535 : g));
}

}  // namespace
}  // namespace ffg

extern "C" size_t minima_workspace_bytes(int64_t n_nodes) {
    if (n_nodes < 0) return 0;
    Carver c(nullptr);
    c.take<int32_t>(size_t(n_nodes));
    c.take<int64_t>(size_t(n_nodes) + 1);
    c.take<int64_t>(size_t(scan_scratch_elems(n_nodes)));
    return c.off;
}

extern "C" ffg_status minima_fraction(const ffg_graph *g, const double *fitness_raw,
                                      double *frac, int64_t *node, void *workspace,
                                      size_t ws_bytes, void *stream_) {
    clear_error();
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (!g || g->n_nodes <= 0 || !g->is_min || !g->node_raw || !fitness_raw || !frac)
        return set_error("graph incomplete, or fitness / frac NULL"), FFG_ERR_INVALID_ARG;
    if (g->n_minima <= 0) return set_error("the graph has no local minimum"), FFG_ERR_EMPTY;
    if (!workspace || !aligned256(workspace))
        return set_error("workspace NULL or not 256-byte aligned"), FFG_ERR_INVALID_ARG;
    const int64_t n = g->n_nodes;
    Carver c(workspace);
    int32_t *flag = c.take<int32_t>(size_t(n));
    int64_t *pos = c.take<int64_t>(size_t(n) + 1);
    int64_t *scratch = c.take<int64_t>(size_t(scan_scratch_elems(n)));
    if (ws_bytes < c.off)
        return set_error("workspace %zu bytes, need %zu", ws_bytes, c.off), FFG_ERR_NO_MEMORY;
    k_min_flags<<<min_grid(n), 256, 0, stream>>>(g->is_min, n, flag);
    count_launch();
    FFG_TRY(check_launch("k_min_flags"));
    FFG_TRY(scan_exclusive(flag, pos, n, scratch, stream));
    k_min_emit<<<min_grid(n), 256, 0, stream>>>(g->is_min, g->node_raw, fitness_raw, pos, n,
                                                g->n_raw, g->f_opt, frac, node);
    count_launch();
    return check_launch("k_min_emit");
}

namespace ffg {
FFG_CHECK_READER(check_read_centrality)
}  // namespace ffg
