// ffg_pagerank.cu -- PageRank centrality on the FFG (Sec. VII-B), pull form.
//
// The matrix of Sec. VII-B is the adjacency matrix with every column scaled
// to sum to one, A[v,u] = 1/outdeg(u) for u -> v.  On an FFG (a DAG) A is
// nilpotent, so the damped form with uniform teleport and uniform
// redistribution of the mass of nodes without out-edges is used:
//   x'[v] = alpha * sum_{u in in(v)} w[u] + (alpha * D + 1 - alpha) / N,
//   w[u]  = x[u] / outdeg[u],   D = sum_{outdeg(u) = 0} x[u].
//
// Two launches per solve.
//
// k_pr_layout builds, in the workspace, a gather-friendly copy of the
// in-edges.  Rows are grouped in tiles of 32 consecutive nodes; a tile's
// in-edges are ordered by (src - dst, dst), i.e. grouped by neighbourhood
// offset.  For an FFG a tile has few distinct offsets (about one per stencil
// slot of the Hamming or adjacent neighbourhood) and each group holds
// consecutive sources, so 32 consecutive entries (a chunk, one per lane)
// gather few 32-byte sectors.  No sort is needed: each row's list is already
// ascending, so a warp merge over the distinct offsets emits the groups in
// order.  Each entry carries the shared-memory offset of its accumulator:
// slot = number of earlier entries of the same chunk with the same row, and
// the accumulator of (slot, row) lives at (slot << 5) | (row ^ slot) (the
// XOR spreads one row's slots over distinct banks).  Within a chunk no two
// lanes share an accumulator and the summation order is fixed.  Entry =
// (src << 8) | offset; padding entries gather node 0 into a dummy slot.
// Tile t's chunks start at chunk floor(in_ptr[32t] / 32) + t.  Tiles that do
// not fit (more than kSortCap edges, a row with more than kMaxSlots entries
// in one chunk, or 2^24 nodes and more) keep the plain CSR path.
//
// k_pagerank is one cooperative persistent launch for every iteration.
// Each block owns a contiguous range of tiles of about equal cost and its
// warps take tiles from it in turn; lane t owns row 32*tile + t, so per-row
// loads and stores are coalesced.  One
// lane streams the tile's chunks into a double-buffered shared-memory stage
// with TMA bulk copies (cp.async.bulk, completion on an mbarrier), one
// segment ahead, while the warp gathers w for the current segment and adds
// into its accumulators.  Only w is kept between iterations (ping-pong):
// x[v] = w[v] * outdeg[v] (or w[v] for a node without out-edges).  Residual
// sum |x'-x|, next D and sum x' are accumulated as exact 64-bit fixed-point
// integers (quantum 2^-60), reduced per block into a double-buffered
// partials array, and after a grid barrier every block sums the partials;
// integer sums do not depend on order, so all blocks take the same stopping
// decision and results are deterministic however tiles were scheduled.
// Every wait (grid barrier, mbarrier) is bounded; on expiry the kernel
// records FFG_ERR_TIMEOUT, lets its own copies land, and returns.
#include "ffg_internal.cuh"

namespace ffg {

namespace {

constexpr int kPrThreads = 256;
constexpr int kWarps = kPrThreads / 32;
constexpr int kMaxBlocks = 4096;
constexpr uint64_t kTimeoutNs = 2000000000ULL;
constexpr int kSortCap = 2048;          // in-edges per tile staged by the layout kernel
constexpr int kMaxSlots = 7;            // entries of one row within one chunk
constexpr uint32_t kDummyOff = (7u << 5) | 7u;  // accumulator of padding entries
constexpr uint32_t kPadEntry = kDummyOff;       // source 0, dummy accumulator
constexpr int kAccElems = 8 * 32;       // accumulators per warp (7 slots + dummy)
#ifndef FFG_PR_SEG
#define FFG_PR_SEG 16
#endif
#ifndef FFG_PR_GROUP
#define FFG_PR_GROUP 8
#endif
#ifndef FFG_PR_MINBLOCKS
#define FFG_PR_MINBLOCKS 3
#endif
constexpr int kSeg = FFG_PR_SEG;        // chunks per TMA segment
constexpr int kGroup = FFG_PR_GROUP;    // gathers in flight per lane
constexpr int64_t kMaxPackedNodes = int64_t(1) << 24;
constexpr int kLayoutThreads = 64;
constexpr int64_t kRowCost = 20;        // per-row cost in in-edge units (block split)

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
    long long *partials;  // [2][kMaxBlocks][4] fixed-point block sums
    void *w0, *w1;
    uint32_t *layout;  // packed chunks
    uint8_t *meta;     // per tile: accumulator slots used (1..kMaxSlots), 0 = CSR path
    size_t bytes;
};

inline int64_t layout_chunks(int64_t n, int64_t e) { return e / 32 + (n + 31) / 32 + 1; }

PrWs carve(void *base, int64_t n, int64_t e, size_t elem) {
    Carver c(base);
    PrWs w;
    w.ctl = c.take<PrCtl>(1);
    w.partials = c.take<long long>(size_t(2) * kMaxBlocks * 4);
    w.w0 = c.take<char>(size_t(n) * elem);
    w.w1 = c.take<char>(size_t(n) * elem);
    w.layout = c.take<uint32_t>(size_t(layout_chunks(n, e)) * 32);
    w.meta = c.take<uint8_t>(size_t((n + 31) / 32));
    w.bytes = c.off;
    return w;
}

// ---------------------------------------------------------------------------
// synchronisation primitives (all waits bounded)
// ---------------------------------------------------------------------------
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
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// one lane: expect `bytes` on `bar` and start the bulk copy global -> shared
__device__ __forceinline__ void tma_load(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "{\n .reg .b64 state;\n mbarrier.arrive.expect_tx.shared::cta.b64 state, [%0], %1;\n}" ::
            "r"(smem_addr(bar)),
        "r"(bytes)
        : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the completion of phase `parity`; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    for (uint32_t polls = 0;; ++polls) {
        if (mbar_try_wait(bar, parity)) return true;
        if (polls > (1u << 22) || global_ns() - t0 > kTimeoutNs) return false;
    }
}

// Barrier over the `group` blocks of one job (all co-resident: cooperative
// launch).  Bounded: gives up after
// kTimeoutNs (or 2^24 polls), records FFG_ERR_TIMEOUT.  Returns false
// (uniformly for the whole block) if the run must stop.
__device__ bool group_barrier(PrCtl *ctl, unsigned target, int group) {
    __shared__ int s_ok;
    __syncthreads();
    if (group == 1) return true;  // a one-block group only needs the block barrier
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

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------

// The residual, the dangling mass and the sum of x are accumulated as 64-bit
// fixed-point integers with quantum 2^-60 (all three are sums of
// non-negative values below 8).  Integer sums are exact and independent of
// order, so they are deterministic however tiles are scheduled, and they use
// no FP64 instruction (a narrow pipe on this part) on the per-row path.
constexpr double kFix = 1152921504606846976.0;  // 2^60
__device__ __forceinline__ long long to_fix(float x) {
    return __float2ll_rn(x * 1152921504606846976.0f);
}
__device__ __forceinline__ long long to_fix(double x) { return __double2ll_rn(x * kFix); }

struct Fix3 {
    long long r = 0, d = 0, s = 0;
};

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block sums of the three accumulators; valid in thread 0
__device__ __forceinline__ Fix3 block_sum_fix(Fix3 v) {
    __shared__ long long red[3][kWarps];
    v.r = warp_sum_ll(v.r);
    v.d = warp_sum_ll(v.d);
    v.s = warp_sum_ll(v.s);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        red[0][warp] = v.r;
        red[1][warp] = v.d;
        red[2][warp] = v.s;
    }
    __syncthreads();
    Fix3 t;
    if (threadIdx.x == 0)
        for (int k = 0; k < kWarps; ++k) {
            t.r += red[0][k];
            t.d += red[1][k];
            t.s += red[2][k];
        }
    return t;
}

struct Tot {
    double r, d, s;
};

// every block sums the partials of all blocks (warp 0)
__device__ __forceinline__ Tot sum_partials(const long long *part, int nb) {
    __shared__ double s_out[3];
    if (threadIdx.x < 32) {
        long long a = 0, b = 0, c = 0;
        for (int k = threadIdx.x; k < nb; k += 32) {
            a += __ldcg(part + 4 * k + 0);
            b += __ldcg(part + 4 * k + 1);
            c += __ldcg(part + 4 * k + 2);
        }
        a = warp_sum_ll(a);
        b = warp_sum_ll(b);
        c = warp_sum_ll(c);
        if (threadIdx.x == 0) {
            s_out[0] = static_cast<double>(a) / kFix;
            s_out[1] = static_cast<double>(b) / kFix;
            s_out[2] = static_cast<double>(c) / kFix;
        }
    }
    __syncthreads();
    Tot t{s_out[0], s_out[1], s_out[2]};
    __syncthreads();
    return t;
}

// ---------------------------------------------------------------------------
// gather-friendly layout of the in-edges (built once per solve)
// ---------------------------------------------------------------------------
// One tile of the layout (one warp): see the comment at the top of the file.
__device__ void layout_tiles(const int64_t *__restrict__ in_ptr, const int32_t *__restrict__ in_idx,
                             int64_t n, uint32_t *__restrict__ layout, uint8_t *__restrict__ meta,
                             int64_t t, int32_t *src, int lane) {
    const unsigned lt_mask = (1u << lane) - 1u;
    do {
        const int64_t r0 = t << 5;
        const int64_t rend = r0 + 32 < n ? r0 + 32 : n;
        const int64_t ip0 = in_ptr[r0], ip1 = in_ptr[rend];
        const int64_t et = ip1 - ip0;
        if (et > kSortCap || n >= kMaxPackedNodes) {
            if (lane == 0) meta[t] = 0;
            break;
        }
        for (int64_t k = lane; k < et; k += 32) src[k] = in_idx[ip0 + k];
        const int64_t v = r0 + lane;
        int cur = 0, end = 0;
        if (v < rend) {
            cur = static_cast<int>(in_ptr[v] - ip0);
            end = static_cast<int>(in_ptr[v + 1] - ip0);
        }
        __syncwarp();
        const int64_t base = ((ip0 >> 5) + t) * 32;  // first entry of the tile
        int pos = 0, last_chunk = -1, count = 0, maxslot = 0;
        // merge the 32 ascending lists by offset src - dst; one group per offset
        while (true) {
            const int32_t head = cur < end ? src[cur] - static_cast<int32_t>(v) : INT32_MAX;
            int32_t m = head;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const int32_t y = __shfl_xor_sync(0xffffffffu, m, o);
                m = y < m ? y : m;
            }
            if (m == INT32_MAX) break;
            const bool hit = head == m;
            const unsigned mask = __ballot_sync(0xffffffffu, hit);
            if (hit) {
                const int p = pos + __popc(mask & lt_mask);
                const int chunk = p >> 5;
                if (chunk != last_chunk) {
                    last_chunk = chunk;
                    count = 0;
                }
                const int slot = count++;
                if (slot > maxslot) maxslot = slot;
                const uint32_t sl = static_cast<uint32_t>(slot < kMaxSlots ? slot : 0);
                layout[base + p] = (static_cast<uint32_t>(src[cur]) << 8) | (sl << 5) |
                                   (static_cast<uint32_t>(lane) ^ sl);
                ++cur;
            }
            pos += __popc(mask);
        }
        const int padded = (pos + 31) & ~31;
        if (pos + lane < padded) layout[base + pos + lane] = kPadEntry;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int y = __shfl_xor_sync(0xffffffffu, maxslot, o);
            maxslot = y > maxslot ? y : maxslot;
        }
        if (lane == 0) meta[t] = maxslot < kMaxSlots ? static_cast<uint8_t>(maxslot + 1) : 0;
    } while (false);
    __syncwarp();
}

__global__ void __launch_bounds__(kLayoutThreads) k_pr_layout(
    const int64_t *__restrict__ in_ptr, const int32_t *__restrict__ in_idx, int64_t n,
    uint32_t *__restrict__ layout, uint8_t *__restrict__ meta) {
    __shared__ int32_t s_src[kLayoutThreads / 32][kSortCap];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t ntiles = (n + 31) >> 5;
    const int64_t step = int64_t(gridDim.x) * (kLayoutThreads / 32);
    for (int64_t t = int64_t(blockIdx.x) * (kLayoutThreads / 32) + warp; t < ntiles; t += step)
        layout_tiles(in_ptr, in_idx, n, layout, meta, t, s_src[warp], lane);
}

// ---------------------------------------------------------------------------
// per-iteration tile work
// ---------------------------------------------------------------------------
template <typename T>
struct TileInfo {
    int64_t t, e0, e1;  // tile index, in-edge range
    int nslots;         // accumulator slots (0 = CSR path)
    int32_t od;         // out-degree of this lane's row
    T wv;               // w of this lane's row
    __device__ __forceinline__ int nch() const { return static_cast<int>((e1 - e0 + 31) >> 5); }
    __device__ __forceinline__ int64_t chunk0() const { return (e0 >> 5) + t; }
};

template <typename T>
__device__ __forceinline__ TileInfo<T> load_info(int64_t t, int64_t n,
                                                 const int64_t *__restrict__ in_ptr,
                                                 const uint8_t *__restrict__ meta,
                                                 const int32_t *__restrict__ outdeg, const T *wc,
                                                 int lane) {
    TileInfo<T> ti;
    const int64_t r0 = t << 5;
    const int64_t rend = r0 + 32 < n ? r0 + 32 : n;
    const int64_t v = r0 + lane;
    ti.t = t;
    ti.e0 = __ldg(in_ptr + r0);
    ti.e1 = __ldg(in_ptr + rend);
    ti.nslots = __ldg(meta + t);
    ti.od = v < rend ? __ldg(outdeg + v) : 0;
    ti.wv = v < rend ? wc[v] : T(0);
    return ti;
}

// Per-warp TMA stream of packed chunk segments into a two-buffer stage.
// `pending` has bit b set while a copy into buffer b is outstanding.
struct Stream {
    uint32_t *stage;   // [2][kSeg * 32]
    uint64_t *bar;     // [2]
    uint32_t phase;    // bit b = parity of the next completion on buffer b
    uint32_t pending;  // bit b = a copy into buffer b is outstanding
    int buf;           // buffer of the segment to process next
    bool issued;       // the segment for `buf` has been issued
    __device__ __forceinline__ void issue(const uint32_t *layout, int64_t chunk, int cnt, int b,
                                          int lane) {
        if (lane == 0) {
            tma_load(stage + b * (kSeg * 32), layout + chunk * 32, static_cast<uint32_t>(cnt) * 128u,
                     bar + b);
        }
        pending |= 1u << b;
    }
    // bounded wait on buffer b, uniform over the warp; false on timeout
    __device__ __forceinline__ bool wait(int b) {
        const bool ok = __all_sync(0xffffffffu, mbar_wait(bar + b, (phase >> b) & 1u));
        if (ok) {
            phase ^= 1u << b;
            pending &= ~(1u << b);
        }
        return ok;
    }
    // after a failure: let every outstanding copy of this warp land (bounded)
    __device__ __forceinline__ void drain() {
        for (int b = 0; b < 2; ++b)
            if (pending & (1u << b)) wait(b);
    }
};

// Sum over the rows of a packed tile (lane = row), streaming its chunks in
// segments of kSeg; the segment after the current one (or the first segment
// of the next tile) is copied while the current one is gathered.
template <typename T>
__device__ __forceinline__ bool tile_sum_packed(const uint32_t *__restrict__ layout,
                                                const TileInfo<T> &cur, const TileInfo<T> &nxt,
                                                bool has_next, Stream &st, const T *wc, T *acc,
                                                int lane, T &sum) {
    const int nch = cur.nch();
    for (int k = 0; k < cur.nslots; ++k) acc[(k << 5) | (lane ^ k)] = T(0);
    __syncwarp();
    const int nseg = (nch + kSeg - 1) / kSeg;
    const bool next_packed = has_next && nxt.nslots > 0 && nxt.nch() > 0;
    for (int s = 0; s < nseg; ++s) {
        const int c0 = s * kSeg;
        const int cnt = nch - c0 < kSeg ? nch - c0 : kSeg;
        if (!st.issued) st.issue(layout, cur.chunk0() + c0, cnt, st.buf, lane);
        // prefetch the following segment into the other buffer
        if (s + 1 < nseg) {
            const int c1 = c0 + kSeg;
            st.issue(layout, cur.chunk0() + c1, nch - c1 < kSeg ? nch - c1 : kSeg, st.buf ^ 1,
                     lane);
            st.issued = true;
        } else if (next_packed) {
            const int n1 = nxt.nch();
            st.issue(layout, nxt.chunk0(), n1 < kSeg ? n1 : kSeg, st.buf ^ 1, lane);
            st.issued = true;
        } else {
            st.issued = false;
        }
        if (!st.wait(st.buf)) return false;
        const uint32_t *ent = st.stage + st.buf * (kSeg * 32) + lane;
        for (int g0 = 0; g0 < cnt; g0 += kGroup) {
            uint32_t e[kGroup];
            T val[kGroup];
#pragma unroll
            for (int g = 0; g < kGroup; ++g) e[g] = g0 + g < cnt ? ent[(g0 + g) * 32] : kPadEntry;
#pragma unroll
            for (int g = 0; g < kGroup; ++g) val[g] = wc[e[g] >> 8];
#pragma unroll
            for (int g = 0; g < kGroup; ++g) {
                acc[e[g] & 0xffu] += val[g];
                __syncwarp();
            }
        }
        st.buf ^= 1;
    }
    if (nseg == 0 && !st.issued && next_packed) {
        const int n1 = nxt.nch();
        st.issue(layout, nxt.chunk0(), n1 < kSeg ? n1 : kSeg, st.buf, lane);
        st.issued = true;
    }
    T s = T(0);
    for (int k = 0; k < cur.nslots; ++k) s += acc[(k << 5) | (lane ^ k)];
    __syncwarp();
    sum = s;
    return true;
}

// CSR path of one tile: the tile's in-edges [e0, e1) are streamed in windows
// with coalesced in_idx loads, gathered into shared memory, and each lane
// adds the part of its own row [p, p_next) that lies in the window.
template <typename T>
__device__ __forceinline__ T tile_sum_csr(const int32_t *__restrict__ in_idx, const T *wc,
                                          T *buf, int64_t p, int64_t p_next, int64_t e0,
                                          int64_t e1, int lane) {
    T s = T(0);
    for (int64_t ws = e0; ws < e1; ws += kAccElems) {
        const int n = static_cast<int>(e1 - ws < kAccElems ? e1 - ws : kAccElems);
        const int32_t *src = in_idx + ws;
        int i = lane;
        for (; i + 96 < n; i += 128) {
            const int32_t j0 = __ldg(src + i), j1 = __ldg(src + i + 32);
            const int32_t j2 = __ldg(src + i + 64), j3 = __ldg(src + i + 96);
            const T a0 = wc[j0], a1 = wc[j1], a2 = wc[j2], a3 = wc[j3];
            buf[i] = a0;
            buf[i + 32] = a1;
            buf[i + 64] = a2;
            buf[i + 96] = a3;
        }
        for (; i < n; i += 32) buf[i] = wc[__ldg(src + i)];
        __syncwarp();
        const int64_t a = p > ws ? p : ws;
        const int64_t b = p_next < ws + n ? p_next : ws + n;
        for (int64_t e = a; e < b; ++e) s += buf[e - ws];
        __syncwarp();
    }
    return s;
}

// First tile of part w when the tiles are split into nw contiguous ranges of
// about equal cost (in-edges plus kRowCost per row).
__device__ __forceinline__ int64_t tile_split(const int64_t *__restrict__ in_ptr, int64_t n,
                                              int64_t ntiles, int64_t w, int64_t nw) {
    if (w <= 0) return 0;
    if (w >= nw) return ntiles;
    const int64_t total = __ldg(in_ptr + n) + kRowCost * n;
    const int64_t target = total / nw * w + (total % nw) * w / nw;
    int64_t lo = 0, hi = ntiles;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int64_t r = mid << 5 < n ? mid << 5 : n;
        if (__ldg(in_ptr + r) + kRowCost * r >= target) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

template <typename T>
constexpr size_t pr_smem_bytes() {
    return size_t(kWarps) * (2 * kSeg * 32 * sizeof(uint32_t) + kAccElems * sizeof(T) + 16);
}

// One PageRank job: a graph, its layout, its buffers and its parameters.
// `group` blocks work on it together (ranks 0..group-1), synchronised by the
// job's own bounded barrier in `ctl`.
struct JobDev {
    const int64_t *in_ptr;
    const int32_t *in_idx;
    const int32_t *outdeg;
    const uint32_t *layout;
    const uint8_t *meta;
    void *ranks, *w0, *w1;
    long long *partials;  // [2][group][4]
    PrCtl *ctl;
    int64_t n;
    double alpha, tol;
    int max_iter, init, group, pad;
};

// A group of blocks runs all iterations of one job.  Returns false if the
// block must stop (a bounded wait expired).
template <typename T>
__device__ bool run_job(const JobDev &J, int rank, Stream &st, T *acc) {
    const int64_t *__restrict__ in_ptr = J.in_ptr;
    const int32_t *__restrict__ in_idx = J.in_idx;
    const int32_t *__restrict__ outdeg = J.outdeg;
    const uint32_t *__restrict__ layout = J.layout;
    const uint8_t *__restrict__ meta = J.meta;
    const int64_t n = J.n;
    const int nb = J.group;
    T *ranks = static_cast<T *>(J.ranks);
    T *w0 = static_cast<T *>(J.w0), *w1 = static_cast<T *>(J.w1);
    long long *partials = J.partials;
    PrCtl *ctl = J.ctl;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    const int64_t ntiles = (n + 31) >> 5;
    // the block's contiguous tile range (about equal cost per block); its
    // warps take tiles from it in turn through a shared counter
    __shared__ int64_t s_range[2];
    __shared__ unsigned long long s_next;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_range[0] = tile_split(in_ptr, n, ntiles, rank, nb);
        s_range[1] = tile_split(in_ptr, n, ntiles, rank + 1, nb);
        s_next = static_cast<unsigned long long>(s_range[0] + kWarps);
    }
    __syncthreads();
    const int64_t bt0 = s_range[0], bt1 = s_range[1];
    const double inv_n = 1.0 / static_cast<double>(n);

    // prologue: w from the start vector, D_0 and sum x_0 (grid-stride)
    {
        Fix3 acc0;
        const int64_t stride = int64_t(nb) * kPrThreads;
        for (int64_t v = int64_t(rank) * kPrThreads + threadIdx.x; v < n; v += stride) {
            const double x0 = J.init ? static_cast<double>(ranks[v]) : inv_n;
            const int32_t od = __ldg(outdeg + v);
            w0[v] = static_cast<T>(od ? x0 / od : x0);
            const long long q = to_fix(x0);
            if (od == 0) acc0.d += q;
            acc0.s += q;
        }
        const Fix3 b = block_sum_fix(acc0);
        if (threadIdx.x == 0) {
            long long *p = partials + 4 * rank;
            p[0] = 0;
            p[1] = b.d;
            p[2] = b.s;
        }
    }
    unsigned phase = 1;
    if (!group_barrier(ctl, phase * nb, nb)) return false;
    Tot tot = sum_partials(partials, nb);
    double dang = tot.d, xs = tot.s;
    double res = __longlong_as_double(0x7ff0000000000000LL), prev_res = res;
    int it = 0, converged = 0;
    T *wc = w0, *wn = w1;
    int par = 0;
    const double alpha = J.alpha;
    const T a = static_cast<T>(alpha);
    int failed = 0;
    while (true) {
        const T c = static_cast<T>((alpha * dang + 1.0 - alpha) * inv_n);
        Fix3 facc;
        int64_t t = bt0 + warp;
        if (t < bt1 && !failed) {
            TileInfo<T> cur = load_info<T>(t, n, in_ptr, meta, outdeg, wc, lane);
            while (true) {
                unsigned long long g = 0;
                if (lane == 0) g = atomicAdd(&s_next, 1ULL);
                const int64_t tn = static_cast<int64_t>(__shfl_sync(0xffffffffu, g, 0));
                const bool has_next = tn < bt1;
                TileInfo<T> nxt = cur;
                if (has_next) nxt = load_info<T>(tn, n, in_ptr, meta, outdeg, wc, lane);
                const int64_t v = (t << 5) + lane;
                const bool row_ok = v < n;
                T s = T(0);
                if (cur.nslots > 0) {
                    if (!tile_sum_packed<T>(layout, cur, nxt, has_next, st, wc, acc, lane, s)) {
                        failed = 1;
                        break;
                    }
                } else {
                    const int64_t p = row_ok ? __ldg(in_ptr + v) : cur.e1;
                    int64_t p_next = __shfl_down_sync(0xffffffffu, p, 1);
                    if (lane == 31 || v + 1 >= n) p_next = cur.e1;
                    // the next packed tile's first segment streams in meanwhile
                    if (!st.issued && has_next && nxt.nslots > 0 && nxt.nch() > 0) {
                        const int n1 = nxt.nch();
                        st.issue(layout, nxt.chunk0(), n1 < kSeg ? n1 : kSeg, st.buf, lane);
                        st.issued = true;
                    }
                    s = tile_sum_csr<T>(in_idx, wc, acc, p, p_next, cur.e0, cur.e1, lane);
                }
                if (row_ok) {
                    const T xo = cur.od ? cur.wv * static_cast<T>(cur.od) : cur.wv;
                    const T xn = a * s + c;
                    facc.r += to_fix(xn > xo ? xn - xo : xo - xn);
                    const long long q = to_fix(xn);
                    if (cur.od == 0) facc.d += q;
                    facc.s += q;
                    wn[v] = cur.od ? xn / static_cast<T>(cur.od) : xn;
                }
                if (!has_next) break;
                cur = nxt;
                t = tn;
            }
        }
        if (failed == 1) {
            // let this warp's own copies land (bounded), then report
            st.drain();
            if (lane == 0) atomicCAS(&ctl->status, 0, (int)FFG_ERR_TIMEOUT);
            failed = 2;
        }
        const Fix3 b = block_sum_fix(facc);
        par ^= 1;
        long long *pp = partials + size_t(par) * nb * 4;
        if (threadIdx.x == 0) {
            long long *p = pp + 4 * rank;
            p[0] = b.r;
            p[1] = b.d;
            p[2] = b.s;
            s_next = static_cast<unsigned long long>(bt0 + kWarps);  // next iteration's counter
        }
        ++phase;
        if (!group_barrier(ctl, phase * nb, nb)) return false;
        tot = sum_partials(pp, nb);
        prev_res = res;
        res = tot.r;
        dang = tot.d;
        xs = tot.s;
        ++it;
        T *tmp = wc;
        wc = wn;
        wn = tmp;
        if (res < J.tol) { converged = 1; break; }
        if (sizeof(T) == 4 && res >= prev_res) { converged = 1; break; }  // FP32 rounding floor
        if (it >= J.max_iter) break;
    }
    // epilogue: x' normalised to sum 1
    const double inv_s = 1.0 / xs;
    const int64_t stride = int64_t(nb) * kPrThreads;
    for (int64_t v = int64_t(rank) * kPrThreads + threadIdx.x; v < n; v += stride) {
        const int32_t od = __ldg(outdeg + v);
        const double x = od ? static_cast<double>(wc[v]) * od : static_cast<double>(wc[v]);
        ranks[v] = static_cast<T>(x * inv_s);
    }
    if (rank == 0 && threadIdx.x == 0) {
        ctl->iters = it;
        ctl->residual = res;
        ctl->converged = converged;
        ctl->nblocks = nb;
    }
    return failed == 0;
}

// The persistent kernel.  With jobs == nullptr it runs `single` on the whole
// grid; otherwise block b runs the plan items [first[b], first[b+1]) in
// order -- (job, rank) pairs, each block's multi-block job first, so that
// no two groups ever wait on each other.
template <typename T>
__global__ void __launch_bounds__(kPrThreads, FFG_PR_MINBLOCKS)
    k_pagerank(const JobDev *__restrict__ jobs, const int2 *__restrict__ items,
               const int *__restrict__ first, int plan_blocks, JobDev single) {
    extern __shared__ __align__(128) unsigned char s_dyn[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // shared memory: per-warp stages, then accumulators, then mbarriers
    Stream st;
    st.stage = reinterpret_cast<uint32_t *>(s_dyn) + size_t(warp) * 2 * kSeg * 32;
    T *acc = reinterpret_cast<T *>(s_dyn + size_t(kWarps) * 2 * kSeg * 32 * sizeof(uint32_t)) +
             size_t(warp) * kAccElems;
    st.bar = reinterpret_cast<uint64_t *>(s_dyn + size_t(kWarps) * 2 * kSeg * 32 * sizeof(uint32_t) +
                                          size_t(kWarps) * kAccElems * sizeof(T)) +
             2 * warp;
    st.phase = 0;
    st.pending = 0;
    st.buf = 0;
    st.issued = false;
    if (lane == 0) {
        mbar_init(st.bar);
        mbar_init(st.bar + 1);
        fence_mbar_init();
    }
    __syncwarp();
    if (jobs == nullptr) {
        run_job<T>(single, blockIdx.x, st, acc);
        return;
    }
    if (static_cast<int>(gridDim.x) != plan_blocks) return;  // the host checks this too
    for (int i = first[blockIdx.x]; i < first[blockIdx.x + 1]; ++i) {
        const int2 item = items[i];
        const JobDev J = jobs[item.x];
        if (!run_job<T>(J, item.y, st, acc)) return;
    }
}

// Layout kernel over every distinct graph of a batch: global tile index ->
// graph by binary search over the graphs' first tiles.
struct GraphDev {
    const int64_t *in_ptr;
    const int32_t *in_idx;
    uint32_t *layout;
    uint8_t *meta;
    int64_t n;
    int64_t tile0;  // first global tile of this graph
};

__global__ void __launch_bounds__(kLayoutThreads) k_pr_layout_batch(const GraphDev *__restrict__ gr,
                                                                     int n_graphs,
                                                                     int64_t total_tiles) {
    __shared__ int32_t s_src[kLayoutThreads / 32][kSortCap];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t step = int64_t(gridDim.x) * (kLayoutThreads / 32);
    for (int64_t gt = int64_t(blockIdx.x) * (kLayoutThreads / 32) + warp; gt < total_tiles;
         gt += step) {
        int lo = 0, hi = n_graphs - 1;  // last graph with tile0 <= gt
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (gr[mid].tile0 <= gt) lo = mid;
            else hi = mid - 1;
        }
        const GraphDev g = gr[lo];
        layout_tiles(g.in_ptr, g.in_idx, g.n, g.layout, g.meta, gt - g.tile0, s_src[warp], lane);
    }
}

ffg_status launch_layout(const ffg_graph *g, PrWs &w, cudaStream_t stream) {
    int dev = 0, sms = 0;
    FFG_TRY(check_cuda(cudaGetDevice(&dev), "cudaGetDevice"));
    FFG_TRY(check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "attr"));
    const int64_t n = g->n_nodes;
    const int64_t tiles = (n + 31) / 32;
    const int64_t want = (tiles + kLayoutThreads / 32 - 1) / (kLayoutThreads / 32);
    const int64_t cap = int64_t(sms) * 32;
    const unsigned grid = static_cast<unsigned>(want < cap ? want : cap);
    k_pr_layout<<<grid, kLayoutThreads, 0, stream>>>(g->in_ptr, g->in_idx, n, w.layout, w.meta);
    count_launch();
    return check_launch("k_pr_layout");
}

template <typename T>
ffg_status kernel_config(int *blocks_per_sm, int *sms) {
    int dev = 0;
    FFG_TRY(check_cuda(cudaGetDevice(&dev), "cudaGetDevice"));
    FFG_TRY(check_cuda(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev), "attr"));
    auto kern = k_pagerank<T>;
    const size_t smem = pr_smem_bytes<T>();
    FFG_TRY(check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            static_cast<int>(smem)),
                       "smem attribute"));
    FFG_TRY(check_cuda(
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, kPrThreads, smem),
        "occupancy"));
    if (*blocks_per_sm < 1) return set_error("kernel does not fit on the device"), FFG_ERR_CUDA;
    return FFG_OK;
}

template <typename T>
ffg_status launch_pr(const JobDev *jobs, const int2 *items, const int *first, int nb,
                     const JobDev &single, cudaStream_t stream) {
    auto kern = k_pagerank<T>;
    const size_t smem = pr_smem_bytes<T>();
    JobDev s = single;
    void *args[] = {(void *)&jobs, (void *)&items, (void *)&first, (void *)&nb, (void *)&s};
    FFG_TRY(check_cuda(cudaLaunchCooperativeKernel((const void *)kern, dim3(nb), dim3(kPrThreads),
                                                   args, smem, stream),
                       "k_pagerank"));
    count_launch();
    return FFG_OK;
}

template <typename T>
ffg_status launch(const ffg_graph *g, double alpha, double tol, int max_iter, int init,
                  T *ranks, PrWs &w, cudaStream_t stream) {
    int per_sm = 0, sms = 0;
    FFG_TRY(kernel_config<T>(&per_sm, &sms));
    const int64_t tiles = (g->n_nodes + 31) / 32;
    int64_t max_res = int64_t(sms) * per_sm;
    if (max_res > kMaxBlocks) max_res = kMaxBlocks;
    const int64_t want = (tiles + 4 * kWarps - 1) / (4 * kWarps);  // >= ~4 tiles per warp
    const int nb = static_cast<int>(want < 1 ? 1 : (want > max_res ? max_res : want));
    JobDev J;
    J.in_ptr = g->in_ptr;
    J.in_idx = g->in_idx;
    J.outdeg = g->outdeg;
    J.layout = w.layout;
    J.meta = w.meta;
    J.ranks = ranks;
    J.w0 = w.w0;
    J.w1 = w.w1;
    J.partials = w.partials;
    J.ctl = w.ctl;
    J.n = g->n_nodes;
    J.alpha = alpha;
    J.tol = tol;
    J.max_iter = max_iter;
    J.init = init;
    J.group = nb;
    J.pad = 0;
    return launch_pr<T>(nullptr, nullptr, nullptr, nb, J, stream);
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
        set_error("pagerank: a bounded device wait timed out");
        return static_cast<ffg_status>(h.status);
    }
    return h.converged ? FFG_OK : FFG_ERR_NOT_CONVERGED;
}

}  // namespace

}  // namespace ffg

using namespace ffg;

extern "C" size_t pagerank_workspace_bytes(int64_t n_nodes, int64_t n_edges, ffg_prec prec) {
    if (n_nodes < 0 || n_edges < 0) return 0;
    return carve(nullptr, n_nodes, n_edges, prec == FFG_F32 ? 4 : 8).bytes;
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
    PrWs w = carve(workspace, g->n_nodes, g->n_edges, prec == FFG_F32 ? 4 : 8);
    if (ws_bytes < w.bytes)
        return set_error("workspace %zu bytes, need %zu", ws_bytes, w.bytes), FFG_ERR_NO_MEMORY;
    if (init & ~(FFG_INIT_RANKS | FFG_INIT_LAYOUT))
        return set_error("unknown init flags 0x%x", init), FFG_ERR_INVALID_ARG;
    FFG_TRY(check_cuda(cudaMemsetAsync(w.ctl, 0, sizeof(PrCtl), stream), "memset"));
    if (!(init & FFG_INIT_LAYOUT)) FFG_TRY(launch_layout(g, w, stream));
    const int warm = (init & FFG_INIT_RANKS) ? 1 : 0;
    if (prec == FFG_F64)
        FFG_TRY(launch<double>(g, damping, tol, max_iter, warm, static_cast<double *>(ranks), w,
                               stream));
    else
        FFG_TRY(launch<float>(g, damping, tol, max_iter, warm, static_cast<float *>(ranks), w,
                              stream));
    if (!iters_out && !residual_out) return FFG_OK;
    return read_result(w.ctl, iters_out, residual_out, stream);
}

extern "C" ffg_status pagerank_prepare(const ffg_graph *g, ffg_prec prec, void *workspace,
                                       size_t ws_bytes, void *stream_) {
    clear_error();
    if (!g || g->n_nodes <= 0 || !g->in_ptr || (g->n_edges > 0 && !g->in_idx))
        return set_error("graph is empty or incomplete"), FFG_ERR_INVALID_ARG;
    if (g->n_nodes >= (int64_t(1) << 31)) return set_error("too many nodes"), FFG_ERR_OVERFLOW;
    if (prec != FFG_F64 && prec != FFG_F32)
        return set_error("unknown precision %d", (int)prec), FFG_ERR_INVALID_ARG;
    if (!workspace || !aligned256(workspace))
        return set_error("workspace NULL or not 256-byte aligned"), FFG_ERR_INVALID_ARG;
    PrWs w = carve(workspace, g->n_nodes, g->n_edges, prec == FFG_F32 ? 4 : 8);
    if (ws_bytes < w.bytes)
        return set_error("workspace %zu bytes, need %zu", ws_bytes, w.bytes), FFG_ERR_NO_MEMORY;
    return launch_layout(g, w, static_cast<cudaStream_t>(stream_));
}

extern "C" ffg_status pagerank_query(const void *workspace, int32_t *iters_out,
                                     double *residual_out, void *stream_) {
    clear_error();
    if (!workspace || !aligned256(workspace))
        return set_error("workspace NULL or misaligned"), FFG_ERR_INVALID_ARG;
    const PrCtl *ctl = static_cast<const PrCtl *>(workspace);
    return read_result(ctl, iters_out, residual_out, static_cast<cudaStream_t>(stream_));
}

// ---------------------------------------------------------------------------
// batched PageRank: many jobs (graph, damping, tolerance) in one persistent
// launch.  The plan assigns each job a group of blocks: jobs costing more
// than two blocks' share of the total get dedicated blocks (their first
// item on every one of them), the others run on one block each, placed by
// longest-processing-time-first on the least loaded block.
// ---------------------------------------------------------------------------
#include <algorithm>
#include <cmath>
#include <numeric>
#include <queue>
#include <unordered_map>
#include <vector>

namespace ffg {
namespace {

struct PlanHost {
    int nb = 0;
    std::vector<int> group;           // per job
    std::vector<int> first;           // nb + 1
    std::vector<int2> items;          // (job, rank)
    std::vector<int> graph_of_job;    // job -> distinct graph index
    std::vector<const ffg_graph *> graphs;
};

double est_iters(double alpha) { return std::log(1.0 / (1 << 21)) / std::log(alpha); }

ffg_status check_job(const ffg_pr_job &j, int idx) {
    const ffg_graph *g = j.g;
    if (!g || g->n_nodes <= 0 || !g->in_ptr || !g->outdeg || (g->n_edges > 0 && !g->in_idx) ||
        !j.ranks)
        return set_error("job %d: graph empty or incomplete, or ranks NULL", idx),
               FFG_ERR_INVALID_ARG;
    if (g->n_nodes >= (int64_t(1) << 31))
        return set_error("job %d: too many nodes", idx), FFG_ERR_OVERFLOW;
    if (!(j.damping > 0.0 && j.damping < 1.0) || !(j.tol >= 0.0) || j.max_iter < 1 ||
        (j.init & ~FFG_INIT_RANKS))
        return set_error("job %d: bad damping, tol, max_iter or init", idx), FFG_ERR_INVALID_ARG;
    return FFG_OK;
}

ffg_status make_plan(const ffg_pr_job *jobs, int n_jobs, int nb_max, const ffg_pr_tuning &tu,
                     PlanHost &P) {
    // distinct graphs (jobs may share one)
    std::unordered_map<const int64_t *, int> gidx;
    P.graph_of_job.resize(n_jobs);
    std::vector<double> cost(n_jobs);
    int64_t useful = 0;
    for (int j = 0; j < n_jobs; ++j) {
        FFG_TRY(check_job(jobs[j], j));
        const ffg_graph *g = jobs[j].g;
        auto it = gidx.find(g->in_ptr);
        if (it == gidx.end()) {
            it = gidx.emplace(g->in_ptr, static_cast<int>(P.graphs.size())).first;
            P.graphs.push_back(g);
        } else if (P.graphs[it->second]->n_nodes != g->n_nodes ||
                   P.graphs[it->second]->n_edges != g->n_edges) {
            return set_error("jobs %d: two graphs share in_ptr with different sizes", j),
                   FFG_ERR_INVALID_ARG;
        }
        P.graph_of_job[j] = it->second;
        cost[j] = double(g->n_edges + kRowCost * g->n_nodes) * est_iters(jobs[j].damping);
        const int64_t tiles = (g->n_nodes + 31) / 32;
        useful += std::max<int64_t>(1, (tiles + 4 * kWarps - 1) / (4 * kWarps));
    }
    int cap = nb_max;
    if (tu.max_blocks > 0 && tu.max_blocks < cap) cap = tu.max_blocks;
    const int nb = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(cap, useful)));
    P.nb = nb;
    const double total = std::accumulate(cost.begin(), cost.end(), 0.0);
    const double share = total / nb;
    std::vector<int> order(n_jobs);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    P.group.assign(n_jobs, 1);
    std::vector<std::vector<int2>> per_block(nb);
    std::vector<double> load(nb, 0.0);
    int next_block = 0;
    std::vector<int> small;
    for (int j : order) {
        const int64_t tiles = (jobs[j].g->n_nodes + 31) / 32;
        // a job above `split` shares gets about one block per `grain` shares
        int k = cost[j] > tu.split * share
                    ? static_cast<int>(std::llround(cost[j] / (tu.grain * share)))
                    : 1;
        k = static_cast<int>(std::min<int64_t>(k, std::max<int64_t>(1, tiles / kWarps)));
        k = std::min(k, nb - next_block);
        if (k >= 2) {
            P.group[j] = k;
            for (int r = 0; r < k; ++r) {
                per_block[next_block + r].push_back(make_int2(j, r));
                load[next_block + r] += cost[j] / k;
            }
            next_block += k;
        } else {
            small.push_back(j);
        }
    }
    // one-block jobs, longest first, onto the least loaded block
    using Slot = std::pair<double, int>;
    std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
    for (int b = 0; b < nb; ++b) heap.push({load[b], b});
    for (int j : small) {
        Slot s = heap.top();
        heap.pop();
        per_block[s.second].push_back(make_int2(j, 0));
        s.first += cost[j];
        heap.push(s);
    }
    P.first.assign(nb + 1, 0);
    P.items.clear();
    for (int b = 0; b < nb; ++b) {
        P.first[b] = static_cast<int>(P.items.size());
        for (const int2 &it : per_block[b]) P.items.push_back(it);
    }
    P.first[nb] = static_cast<int>(P.items.size());
    return FFG_OK;
}

struct BatchWs {
    JobDev *jobs;
    GraphDev *graphs;
    int *first;
    int2 *items;
    PrCtl *ctl;
    size_t bytes;
};

// Workspace of a plan: tables, then per job ctl / partials / w buffers, then
// per distinct graph the layout and tile metadata.  host_jobs / host_graphs
// (if non-NULL) receive the device pointers of every job and graph.
BatchWs carve_batch(void *base, const ffg_pr_job *jobs, int n_jobs, size_t elem,
                    const PlanHost &P, int nb_max, std::vector<JobDev> *host_jobs,
                    std::vector<GraphDev> *host_graphs) {
    Carver c(base);
    BatchWs w;
    w.jobs = c.take<JobDev>(n_jobs);
    w.graphs = c.take<GraphDev>(P.graphs.size());
    // plan tables sized for any tuning: at most nb_max blocks, and a job in a
    // group of k blocks adds k - 1 items, with sum(k) <= nb_max
    w.first = c.take<int>(size_t(nb_max) + 1);
    w.items = c.take<int2>(size_t(n_jobs) + nb_max);
    w.ctl = c.take<PrCtl>(n_jobs);
    std::vector<GraphDev> gd(P.graphs.size());
    int64_t tile0 = 0;
    for (size_t k = 0; k < P.graphs.size(); ++k) {
        const ffg_graph *g = P.graphs[k];
        gd[k].in_ptr = g->in_ptr;
        gd[k].in_idx = g->in_idx;
        gd[k].layout = c.take<uint32_t>(size_t(layout_chunks(g->n_nodes, g->n_edges)) * 32);
        gd[k].meta = c.take<uint8_t>(size_t((g->n_nodes + 31) / 32));
        gd[k].n = g->n_nodes;
        gd[k].tile0 = tile0;
        tile0 += (g->n_nodes + 31) / 32;
    }
    std::vector<JobDev> jd(n_jobs);
    for (int j = 0; j < n_jobs; ++j) {
        const ffg_graph *g = jobs[j].g;
        const GraphDev &G = gd[P.graph_of_job[j]];
        JobDev &J = jd[j];
        J.in_ptr = g->in_ptr;
        J.in_idx = g->in_idx;
        J.outdeg = g->outdeg;
        J.layout = G.layout;
        J.meta = G.meta;
        J.ranks = jobs[j].ranks;
        J.w0 = c.take<char>(size_t(g->n_nodes) * elem);
        J.w1 = c.take<char>(size_t(g->n_nodes) * elem);
        // sized for any group (<= nb_max): the workspace size does not depend
        // on the tuning
        J.partials = c.take<long long>(size_t(2) * nb_max * 4);
        J.ctl = w.ctl + j;
        J.n = g->n_nodes;
        J.alpha = jobs[j].damping;
        J.tol = jobs[j].tol;
        J.max_iter = jobs[j].max_iter;
        J.init = (jobs[j].init & FFG_INIT_RANKS) ? 1 : 0;
        J.group = P.group[j];
        J.pad = 0;
    }
    w.bytes = c.off;
    if (host_jobs) *host_jobs = std::move(jd);
    if (host_graphs) *host_graphs = std::move(gd);
    return w;
}

ffg_status batch_blocks(ffg_prec prec, int *nb_max) {
    int per_sm = 0, sms = 0;
    if (prec == FFG_F64) FFG_TRY(kernel_config<double>(&per_sm, &sms));
    else FFG_TRY(kernel_config<float>(&per_sm, &sms));
    *nb_max = std::min(kMaxBlocks, sms * per_sm);
    return FFG_OK;
}

}  // namespace
}  // namespace ffg

const ffg_pr_tuning kDefaultTuning = {1.0, 1.0, 0, 0};

extern "C" size_t pagerank_batch_workspace_bytes(const ffg_pr_job *jobs, int32_t n_jobs,
                                                 ffg_prec prec) {
    clear_error();
    if (!jobs || n_jobs < 1 || (prec != FFG_F64 && prec != FFG_F32)) return 0;
    int nb_max = 0;
    if (batch_blocks(prec, &nb_max) != FFG_OK) return 0;
    PlanHost P;
    if (make_plan(jobs, n_jobs, nb_max, kDefaultTuning, P) != FFG_OK) return 0;
    return carve_batch(nullptr, jobs, n_jobs, prec == FFG_F32 ? 4 : 8, P, nb_max, nullptr,
                       nullptr)
        .bytes;
}

extern "C" ffg_status pagerank_batch_plan(const ffg_pr_job *jobs, int32_t n_jobs, ffg_prec prec,
                                          void *workspace, size_t ws_bytes, ffg_pr_batch *plan,
                                          void *stream_) {
    return pagerank_batch_plan_tuned(jobs, n_jobs, prec, &kDefaultTuning, workspace, ws_bytes,
                                     plan, stream_);
}

extern "C" ffg_status pagerank_batch_plan_tuned(const ffg_pr_job *jobs, int32_t n_jobs,
                                                ffg_prec prec, const ffg_pr_tuning *tuning,
                                                void *workspace, size_t ws_bytes,
                                                ffg_pr_batch *plan, void *stream_) {
    clear_error();
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (!jobs || n_jobs < 1 || !plan || !workspace)
        return set_error("jobs, plan and workspace must be non-NULL, n_jobs >= 1"),
               FFG_ERR_INVALID_ARG;
    if (prec != FFG_F64 && prec != FFG_F32)
        return set_error("unknown precision %d", (int)prec), FFG_ERR_INVALID_ARG;
    if (!aligned256(workspace))
        return set_error("workspace not 256-byte aligned"), FFG_ERR_INVALID_ARG;
    const ffg_pr_tuning tu = tuning ? *tuning : kDefaultTuning;
    if (!(tu.split > 0.0) || !(tu.grain > 0.0) || tu.max_blocks < 0)
        return set_error("tuning: split and grain must be > 0, max_blocks >= 0"),
               FFG_ERR_INVALID_ARG;
    int nb_max = 0;
    FFG_TRY(batch_blocks(prec, &nb_max));
    PlanHost P;
    FFG_TRY(make_plan(jobs, n_jobs, nb_max, tu, P));
    std::vector<JobDev> jd;
    std::vector<GraphDev> gd;
    BatchWs w = carve_batch(workspace, jobs, n_jobs, prec == FFG_F32 ? 4 : 8, P, nb_max, &jd, &gd);
    if (ws_bytes < w.bytes)
        return set_error("workspace %zu bytes, need %zu", ws_bytes, w.bytes), FFG_ERR_NO_MEMORY;
    if (P.nb > nb_max || P.items.size() > size_t(n_jobs) + nb_max)
        return set_error("internal: plan exceeds its tables"), FFG_ERR_INVALID_ARG;
    FFG_TRY(check_cuda(cudaMemcpyAsync(w.jobs, jd.data(), sizeof(JobDev) * jd.size(),
                                       cudaMemcpyHostToDevice, stream), "upload jobs"));
    FFG_TRY(check_cuda(cudaMemcpyAsync(w.graphs, gd.data(), sizeof(GraphDev) * gd.size(),
                                       cudaMemcpyHostToDevice, stream), "upload graphs"));
    FFG_TRY(check_cuda(cudaMemcpyAsync(w.first, P.first.data(), sizeof(int) * P.first.size(),
                                       cudaMemcpyHostToDevice, stream), "upload plan"));
    if (!P.items.empty())
        FFG_TRY(check_cuda(cudaMemcpyAsync(w.items, P.items.data(), sizeof(int2) * P.items.size(),
                                           cudaMemcpyHostToDevice, stream), "upload plan"));
    FFG_TRY(check_cuda(cudaStreamSynchronize(stream), "sync plan upload"));
    int64_t tiles = 0;
    for (const ffg_graph *g : P.graphs) tiles += (g->n_nodes + 31) / 32;
    plan->prec = prec;
    plan->n_jobs = n_jobs;
    plan->n_graphs = static_cast<int32_t>(P.graphs.size());
    plan->n_blocks = P.nb;
    plan->total_tiles = tiles;
    plan->jobs = w.jobs;
    plan->graphs = w.graphs;
    plan->items = w.items;
    plan->first = w.first;
    plan->ctl = w.ctl;
    return FFG_OK;
}

extern "C" ffg_status pagerank_batch_run(const ffg_pr_batch *plan, void *stream_) {
    clear_error();
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (!plan || plan->n_jobs < 1 || !plan->jobs || !plan->ctl || plan->n_blocks < 1)
        return set_error("plan is empty"), FFG_ERR_INVALID_ARG;
    const ffg_prec prec = static_cast<ffg_prec>(plan->prec);
    int nb_max = 0;
    FFG_TRY(batch_blocks(prec, &nb_max));
    if (plan->n_blocks > nb_max)
        return set_error("plan made for %d blocks, %d fit", plan->n_blocks, nb_max),
               FFG_ERR_INVALID_ARG;
    FFG_TRY(check_cuda(cudaMemsetAsync(plan->ctl, 0, sizeof(PrCtl) * plan->n_jobs, stream),
                       "memset"));
    int dev = 0, sms = 0;
    FFG_TRY(check_cuda(cudaGetDevice(&dev), "cudaGetDevice"));
    FFG_TRY(check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "attr"));
    const int64_t want = (plan->total_tiles + kLayoutThreads / 32 - 1) / (kLayoutThreads / 32);
    const int64_t cap = int64_t(sms) * 32;
    k_pr_layout_batch<<<static_cast<unsigned>(std::max<int64_t>(1, std::min(want, cap))),
                        kLayoutThreads, 0, stream>>>(static_cast<const GraphDev *>(plan->graphs),
                                                     plan->n_graphs, plan->total_tiles);
    count_launch();
    FFG_TRY(check_launch("k_pr_layout_batch"));
    JobDev none{};
    const JobDev *jobs = static_cast<const JobDev *>(plan->jobs);
    const int2 *items = static_cast<const int2 *>(plan->items);
    const int *first = static_cast<const int *>(plan->first);
    if (prec == FFG_F64) return launch_pr<double>(jobs, items, first, plan->n_blocks, none, stream);
    return launch_pr<float>(jobs, items, first, plan->n_blocks, none, stream);
}

extern "C" ffg_status pagerank_batch_query(const ffg_pr_batch *plan, int32_t *iters_out,
                                           double *residual_out, int32_t *status_out,
                                           void *stream_) {
    clear_error();
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (!plan || plan->n_jobs < 1 || !plan->ctl) return set_error("plan is empty"), FFG_ERR_INVALID_ARG;
    std::vector<PrCtl> h(plan->n_jobs);
    FFG_TRY(check_cuda(cudaMemcpyAsync(h.data(), plan->ctl, sizeof(PrCtl) * h.size(),
                                       cudaMemcpyDeviceToHost, stream), "read batch results"));
    FFG_TRY(check_cuda(cudaStreamSynchronize(stream), "sync batch results"));
    ffg_status worst = FFG_OK;
    for (int j = 0; j < plan->n_jobs; ++j) {
        const ffg_status st = h[j].status ? static_cast<ffg_status>(h[j].status)
                                          : (h[j].converged ? FFG_OK : FFG_ERR_NOT_CONVERGED);
        if (iters_out) iters_out[j] = h[j].iters;
        if (residual_out) residual_out[j] = h[j].residual;
        if (status_out) status_out[j] = st;
        if (st == FFG_ERR_TIMEOUT || (st != FFG_OK && worst == FFG_OK)) worst = st;
    }
    if (worst == FFG_ERR_TIMEOUT) set_error("pagerank batch: a bounded device wait timed out");
    return worst;
}
