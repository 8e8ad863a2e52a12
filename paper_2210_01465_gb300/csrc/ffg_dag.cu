// ffg_dag.cu -- exact solve on the FFG (Sec. VII-B): the graph has no cycles
// (every edge goes to a strictly smaller key), so
//   y[v] = 1 + d * sum_{u -> v} y[u] / outdeg[u]
// is solved in one pass over the nodes in a topological order.  The pass
// runs level by level (Kahn's order): a level is the set of nodes whose
// in-neighbours are all done.  Sources (no in-edges) form the first level;
// when a node is done it counts down the pending in-degree of each of its
// out-neighbours, and the one that brings a count to zero queues that
// neighbour for the next level.  The number of levels is the longest
// improving path + 1.
//
// One cooperative persistent launch: every level is a grid-stride pass of
// warps over the current queue, then a bounded grid barrier (FFG_ERR_TIMEOUT
// on expiry).  One warp per queued node: the lanes gather and divide 32
// in-neighbours at a time and the terms are added one by one in CSR order
// (FP64, one rounding per operation, no fused multiply-add), so y does not
// depend on the schedule and equals the sequential solve bit for bit; the
// lanes then count down 32 out-neighbours at a time and queue, with one
// atomic per warp, those that became ready.
// Values written at earlier levels by other blocks are read through L2
// (ld.cg), never from a possibly stale L1 line.
#include "ffg_internal.cuh"

namespace ffg {

namespace {

constexpr int kDagThreads = 256;
constexpr int kDagMaxBlocks = 4096;
constexpr uint64_t kDagTimeoutNs = 2000000000ULL;

struct DagCtl {
    unsigned int barrier;
    int status;
    int levels;
    int pad;
    unsigned int tail[3];  // queue lengths, rotating: current, next, cleared
    unsigned int pad2;
};

struct DagWs {
    DagCtl *ctl;
    int32_t *remaining;  // pending in-degree
    int32_t *q0, *q1;    // level queues
    double *part;        // per-block partial sums (normalisation)
    size_t bytes;
};

DagWs carve_dag(void *base, int64_t n) {
    Carver c(base);
    DagWs w;
    w.ctl = c.take<DagCtl>(1);
    w.remaining = c.take<int32_t>(size_t(n));
    w.q0 = c.take<int32_t>(size_t(n));
    w.q1 = c.take<int32_t>(size_t(n));
    w.part = c.take<double>(kDagMaxBlocks);
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

// Bounded grid barrier (all blocks co-resident: cooperative launch);
// uniform false for the whole block if the run must stop.
__device__ bool dag_barrier(DagCtl *ctl, unsigned target) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        red_release_add(&ctl->barrier, 1u);
        const uint64_t t0 = global_ns();
        unsigned ns = 0;
        int ok = 1;
        for (uint32_t polls = 0; ld_acquire(&ctl->barrier) < target; ++polls) {
            if ((polls & 15) == 15 && *(volatile int *)&ctl->status != 0) {
                ok = 0;
                break;
            }
            if (polls > (1u << 24) || global_ns() - t0 > kDagTimeoutNs) {
                atomicCAS(&ctl->status, 0, (int)FFG_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            if (polls > 64) {
                __nanosleep(ns);
                ns = ns < 32 ? 32 : (ns < 256 ? ns << 1 : ns);
            }
        }
        if (*(volatile int *)&ctl->status != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Neumaier-compensated sum in thread 0 of the block's values
__device__ double block_sum_comp(double v, double c) {
    __shared__ double s_v[kDagThreads / 32], s_c[kDagThreads / 32];
    // warp: pairwise two-sum of (v, c) pairs in a fixed order
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, v, o);
        const double oc = __shfl_down_sync(0xffffffffu, c, o);
        const double t = __dadd_rn(v, ov);
        const double e = fabs(v) >= fabs(ov) ? __dadd_rn(__dadd_rn(v, -t), ov)
                                             : __dadd_rn(__dadd_rn(ov, -t), v);
        v = t;
        c = __dadd_rn(__dadd_rn(c, oc), e);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        s_v[warp] = v;
        s_c[warp] = c;
    }
    __syncthreads();
    double sum = 0.0, comp = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < kDagThreads / 32; ++k) {
            const double t = __dadd_rn(sum, s_v[k]);
            comp = __dadd_rn(comp, fabs(sum) >= fabs(s_v[k]) ? __dadd_rn(__dadd_rn(sum, -t), s_v[k])
                                                             : __dadd_rn(__dadd_rn(s_v[k], -t), sum));
            comp = __dadd_rn(comp, s_c[k]);
            sum = t;
        }
    return __dadd_rn(sum, comp);  // valid in thread 0
}

struct DagArgs {
    const int64_t *in_ptr, *out_ptr;
    const int32_t *in_idx, *out_idx, *outdeg;
    int64_t n;
    double d;
    int mode;
    double *y;
    DagWs w;
};

__global__ void __launch_bounds__(kDagThreads) k_dag(DagArgs a) {
    const int64_t n = a.n;
    const int nb = gridDim.x;
    const int64_t stride = int64_t(nb) * kDagThreads;
    const int64_t gid = int64_t(blockIdx.x) * kDagThreads + threadIdx.x;
    DagCtl *ctl = a.w.ctl;
    int32_t *q[2] = {a.w.q0, a.w.q1};
    // sources form the first level
    for (int64_t v = gid; v < n; v += stride) {
        const int32_t r = static_cast<int32_t>(a.in_ptr[v + 1] - a.in_ptr[v]);
        a.w.remaining[v] = r;
        if (r == 0) q[0][atomicAdd(&ctl->tail[0], 1u)] = static_cast<int32_t>(v);
    }
    unsigned phase = 1;
    if (!dag_barrier(ctl, phase * nb)) return;
    int level = 0;
    while (true) {
        const int cur = level % 3, nxt = (level + 1) % 3, clr = (level + 2) % 3;
        const unsigned F = __ldcg(&ctl->tail[cur]);
        if (F == 0) break;  // the same for every block
        if (blockIdx.x == 0 && threadIdx.x == 0) ctl->tail[clr] = 0;  // used as `nxt` next level
        const int32_t *qc = q[level & 1];
        int32_t *qn = q[(level + 1) & 1];
        const int lane = threadIdx.x & 31;
        const int64_t warps = stride >> 5;
        for (int64_t i = gid >> 5; i < F; i += warps) {
            const int32_t v = __ldcg(qc + i);
            const int64_t e0 = a.in_ptr[v], e1 = a.in_ptr[v + 1];
            double s = 0.0;
            for (int64_t b = e0; b < e1; b += 32) {
                double term = 0.0;
                if (b + lane < e1) {
                    const int32_t u = a.in_idx[b + lane];
                    if (FFG_CHECK(u >= 0 && u < n, 301))
                        term = __ddiv_rn(__ldcg(a.y + u), static_cast<double>(a.outdeg[u]));
                }
                const int m = e1 - b < 32 ? static_cast<int>(e1 - b) : 32;
                for (int k = 0; k < m; ++k) s = __dadd_rn(s, __shfl_sync(0xffffffffu, term, k));
            }
            if (lane == 0) a.y[v] = __dadd_rn(1.0, __dmul_rn(a.d, s));
            const int64_t o1 = a.out_ptr[v + 1];
            for (int64_t b = a.out_ptr[v]; b < o1; b += 32) {
                int32_t t = -1;
                bool ready = false;
                if (b + lane < o1) {
                    t = a.out_idx[b + lane];
                    ready = FFG_CHECK(t >= 0 && t < n, 302) &&
                            atomicSub(&a.w.remaining[t], 1) == 1;
                }
                const unsigned mask = __ballot_sync(0xffffffffu, ready);
                if (mask) {
                    unsigned pos = 0;
                    if (lane == 0) pos = atomicAdd(&ctl->tail[nxt], static_cast<unsigned>(__popc(mask)));
                    pos = __shfl_sync(0xffffffffu, pos, 0);
                    if (ready) qn[pos + __popc(mask & ((1u << lane) - 1u))] = t;
                }
            }
        }
        ++phase;
        if (!dag_barrier(ctl, phase * nb)) return;
        ++level;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->levels = level;
    if (a.mode == FFG_DAG_VALUES) return;
    if (a.mode == FFG_DAG_ABSORB) {
        const double nd = static_cast<double>(n);
        for (int64_t v = gid; v < n; v += stride) a.y[v] = __ddiv_rn(__ldcg(a.y + v), nd);
        return;
    }
    // PageRank: y / sum y, the sum in a fixed order (contiguous block ranges,
    // then the block partials in rank order)
    const int64_t chunk = (n + nb - 1) / nb;
    const int64_t v0 = int64_t(blockIdx.x) * chunk, v1 = v0 + chunk < n ? v0 + chunk : n;
    double s = 0.0, c = 0.0;
    for (int64_t v = v0 + threadIdx.x; v < v1; v += kDagThreads) {
        const double x = __ldcg(a.y + v);
        const double t = __dadd_rn(s, x);
        c = __dadd_rn(c, fabs(s) >= fabs(x) ? __dadd_rn(__dadd_rn(s, -t), x)
                                             : __dadd_rn(__dadd_rn(x, -t), s));
        s = t;
    }
    const double bs = block_sum_comp(s, c);
    if (threadIdx.x == 0) a.w.part[blockIdx.x] = bs;
    ++phase;
    if (!dag_barrier(ctl, phase * nb)) return;
    __shared__ double s_total;
    if (threadIdx.x == 0) {
        double sum = 0.0, comp = 0.0;
        for (int k = 0; k < nb; ++k) {
            const double x = __ldcg(a.w.part + k);
            const double t = __dadd_rn(sum, x);
            comp = __dadd_rn(comp, fabs(sum) >= fabs(x) ? __dadd_rn(__dadd_rn(sum, -t), x)
                                                         : __dadd_rn(__dadd_rn(x, -t), sum));
            sum = t;
        }
        s_total = __dadd_rn(sum, comp);
    }
    __syncthreads();
    for (int64_t v = gid; v < n; v += stride) a.y[v] = __ddiv_rn(__ldcg(a.y + v), s_total);
}

}  // namespace
}  // namespace ffg

using namespace ffg;

extern "C" size_t dag_workspace_bytes(int64_t n_nodes) {
    if (n_nodes < 0) return 0;
    return carve_dag(nullptr, n_nodes).bytes;
}

extern "C" ffg_status dag_solve(const ffg_graph *g, double damping, ffg_dag_mode mode,
                                double *ranks, void *workspace, size_t ws_bytes,
                                int32_t *levels_out, void *stream_) {
    clear_error();
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (!g || g->n_nodes <= 0 || !g->in_ptr || !g->out_ptr || !g->outdeg ||
        (g->n_edges > 0 && (!g->in_idx || !g->out_idx)))
        return set_error("graph is empty or incomplete"), FFG_ERR_INVALID_ARG;
    if (g->n_nodes >= (int64_t(1) << 31)) return set_error("too many nodes"), FFG_ERR_OVERFLOW;
    if (mode != FFG_DAG_VALUES && mode != FFG_DAG_PAGERANK && mode != FFG_DAG_ABSORB)
        return set_error("unknown mode %d", (int)mode), FFG_ERR_INVALID_ARG;
    if (!(damping >= 0.0 && damping <= 1.0) ||
        (mode == FFG_DAG_PAGERANK && !(damping > 0.0 && damping < 1.0)) ||
        (mode == FFG_DAG_ABSORB && damping != 1.0))
        return set_error("damping out of range for the mode"), FFG_ERR_INVALID_ARG;
    if (!ranks || !workspace || !aligned256(workspace))
        return set_error("ranks NULL, or workspace NULL or not 256-byte aligned"),
               FFG_ERR_INVALID_ARG;
    DagWs w = carve_dag(workspace, g->n_nodes);
    if (ws_bytes < w.bytes)
        return set_error("workspace %zu bytes, need %zu", ws_bytes, w.bytes), FFG_ERR_NO_MEMORY;
    int dev = 0, sms = 0, per_sm = 0;
    FFG_TRY(check_cuda(cudaGetDevice(&dev), "cudaGetDevice"));
    FFG_TRY(check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "attr"));
    FFG_TRY(check_cuda(
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dag, kDagThreads, 0),
        "occupancy"));
    if (per_sm < 1) return set_error("k_dag does not fit"), FFG_ERR_CUDA;
    const int64_t want = (g->n_nodes + kDagThreads - 1) / kDagThreads;
    int64_t nb = int64_t(sms) * per_sm;
    if (nb > kDagMaxBlocks) nb = kDagMaxBlocks;
    if (want < nb) nb = want < 1 ? 1 : want;
    FFG_TRY(check_cuda(cudaMemsetAsync(w.ctl, 0, sizeof(DagCtl), stream), "memset"));
    DagArgs a;
    a.in_ptr = g->in_ptr;
    a.out_ptr = g->out_ptr;
    a.in_idx = g->in_idx;
    a.out_idx = g->out_idx;
    a.outdeg = g->outdeg;
    a.n = g->n_nodes;
    a.d = damping;
    a.mode = mode;
    a.y = ranks;
    a.w = w;
    void *args[] = {(void *)&a};
    FFG_TRY(check_cuda(cudaLaunchCooperativeKernel((const void *)k_dag, dim3(unsigned(nb)),
                                                   dim3(kDagThreads), args, 0, stream),
                       "k_dag"));
    count_launch();
    if (!levels_out) return FFG_OK;
    DagCtl h;
    FFG_TRY(check_cuda(cudaMemcpyAsync(&h, w.ctl, sizeof(h), cudaMemcpyDeviceToHost, stream),
                       "read dag result"));
    FFG_TRY(check_cuda(cudaStreamSynchronize(stream), "sync dag"));
    *levels_out = h.levels;
    if (h.status != 0) {
        set_error("dag_solve: a bounded device wait timed out");
        return static_cast<ffg_status>(h.status);
    }
    return FFG_OK;
}

namespace ffg {
FFG_CHECK_READER(check_read_dag)
}  // namespace ffg
