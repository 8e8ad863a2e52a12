// ffg_walk.cu -- simulated improving walks on the FFG (Sec. VII-B: a random
// walk on the FFG mimics a randomised first-improvement local search; the
// PageRank of a minimum is read as the chance of arriving there).
//
// One thread per walk.  Walk j starts at a uniformly random node and moves to
// a uniformly random out-neighbour until it reaches a node without
// out-edges, where it is counted.  Its k-th draw (k = 0 for the start) is the
// k-th output of the SplitMix64 stream (Steele, Lea and Flood, OOPSLA 2014)
// whose state starts at splitmix64(seed ^ j); a draw x picks index
// ((x >> 32) * m) >> 32 among m choices.  Counts are integers added with
// atomics, so they do not depend on the schedule.  On an FFG a walk makes
// fewer than n_nodes moves; a longer one (a graph with a cycle) stops and
// flags FFG_ERR_INVALID_ARG, so every loop is bounded.
#include "ffg_internal.cuh"

namespace ffg {

namespace {

constexpr int kWalkThreads = 256;
constexpr uint64_t kGamma = 0x9e3779b97f4a7c15ULL;

struct WalkCtl {
    unsigned long long steps;
    int status;
    int pad;
};

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + kGamma;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t pick(uint64_t draw, uint64_t m) {
    return ((draw >> 32) * m) >> 32;
}

__global__ void __launch_bounds__(kWalkThreads) k_walks(const int64_t *__restrict__ out_ptr,
                                                        const int32_t *__restrict__ out_idx,
                                                        const int32_t *__restrict__ outdeg,
                                                        int64_t n, uint64_t seed, int64_t n_walks,
                                                        unsigned long long *counts, WalkCtl *ctl) {
    unsigned long long moves = 0;
    for (int64_t j = int64_t(blockIdx.x) * kWalkThreads + threadIdx.x; j < n_walks;
         j += int64_t(gridDim.x) * kWalkThreads) {
        const uint64_t s0 = splitmix64(seed ^ static_cast<uint64_t>(j));
        uint64_t k = 0;
        int64_t v = static_cast<int64_t>(pick(splitmix64(s0), static_cast<uint64_t>(n)));
        int32_t d = __ldg(outdeg + v);
        bool ok = true;
        while (d > 0) {
            if (static_cast<int64_t>(k) >= n) {  // impossible without a cycle
                ok = false;
                break;
            }
            ++k;
            const uint64_t i = pick(splitmix64(s0 + k * kGamma), static_cast<uint64_t>(d));
            v = __ldg(out_idx + __ldg(out_ptr + v) + static_cast<int64_t>(i));
            if (!FFG_CHECK(v >= 0 && v < n, 401)) {
                ok = false;
                break;
            }
            d = __ldg(outdeg + v);
        }
        if (ok) atomicAdd(counts + v, 1ULL);
        else atomicCAS(&ctl->status, 0, (int)FFG_ERR_INVALID_ARG);
        moves += k;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) moves += __shfl_xor_sync(0xffffffffu, moves, o);
    if ((threadIdx.x & 31) == 0 && moves) atomicAdd(&ctl->steps, moves);
}

}  // namespace
}  // namespace ffg

using namespace ffg;

extern "C" size_t walk_workspace_bytes(void) { return 256; }

extern "C" ffg_status walk_simulate(const ffg_graph *g, uint64_t seed, int64_t n_walks,
                                    uint64_t *counts, void *workspace, size_t ws_bytes,
                                    int64_t *steps_out, void *stream_) {
    clear_error();
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (!g || g->n_nodes <= 0 || !g->out_ptr || !g->outdeg || (g->n_edges > 0 && !g->out_idx))
        return set_error("graph is empty or incomplete"), FFG_ERR_INVALID_ARG;
    if (g->n_nodes >= (int64_t(1) << 31)) return set_error("too many nodes"), FFG_ERR_OVERFLOW;
    if (n_walks < 0 || !counts || !workspace || !aligned256(workspace))
        return set_error("n_walks < 0, counts NULL, or workspace NULL / misaligned"),
               FFG_ERR_INVALID_ARG;
    if (ws_bytes < sizeof(WalkCtl)) return set_error("workspace too small"), FFG_ERR_NO_MEMORY;
    WalkCtl *ctl = static_cast<WalkCtl *>(workspace);
    FFG_TRY(check_cuda(cudaMemsetAsync(ctl, 0, sizeof(WalkCtl), stream), "memset"));
    FFG_TRY(check_cuda(cudaMemsetAsync(counts, 0, sizeof(uint64_t) * g->n_nodes, stream),
                       "memset"));
    if (n_walks > 0) {
        int dev = 0, sms = 0;
        FFG_TRY(check_cuda(cudaGetDevice(&dev), "cudaGetDevice"));
        FFG_TRY(check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev),
                           "attr"));
        const int64_t want = (n_walks + kWalkThreads - 1) / kWalkThreads;
        const int64_t cap = int64_t(sms) * 16;
        k_walks<<<static_cast<unsigned>(want < cap ? want : cap), kWalkThreads, 0, stream>>>(
            g->out_ptr, g->out_idx, g->outdeg, g->n_nodes, seed, n_walks,
            reinterpret_cast<unsigned long long *>(counts), ctl);
        count_launch();
        FFG_TRY(check_launch("k_walks"));
    }
    if (!steps_out) return FFG_OK;
    WalkCtl h;
    FFG_TRY(check_cuda(cudaMemcpyAsync(&h, ctl, sizeof(h), cudaMemcpyDeviceToHost, stream),
                       "read walks"));
    FFG_TRY(check_cuda(cudaStreamSynchronize(stream), "sync walks"));
    *steps_out = static_cast<int64_t>(h.steps);
    if (h.status != 0) {
        set_error("walk_simulate: a walk made n_nodes moves (the graph has a cycle)");
        return static_cast<ffg_status>(h.status);
    }
    return FFG_OK;
}

namespace ffg {
FFG_CHECK_READER(check_read_walk)
}  // namespace ffg
