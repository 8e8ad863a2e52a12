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
// k_pr_layout builds, in the workspace, a compact copy of the in-edges.
// Rows are grouped in tiles of 32 consecutive nodes, one row per lane.  In an
// FFG the in-neighbours of a tile lie at few distinct node offsets
// off = src - dst (about one per stencil slot of the Hamming or adjacent
// neighbourhood, a few more where invalid configurations shift the
// numbering), so a tile is stored as a list of descriptors (off, mask): lane
// r has the in-edge (32t + r + off) -> (32t + r) iff bit r of mask is set.
// Eight bytes per descriptor replace four bytes per edge, and the 32 lanes
// of one descriptor gather consecutive sources.  No sort is needed: each
// row's in-list is ascending, so a warp merge over the 32 lists emits the
// offsets in ascending order, and every row sums its in-edges in ascending
// source order.  A tile's list is padded with empty descriptors to a
// multiple of kU and starts at desc_begin(in_ptr[32t], t), which leaves room
// for one descriptor per in-edge; the padded count is kept per tile.
//
// k_pagerank is one cooperative persistent launch for every iteration.
// Each block owns a contiguous range of tiles of about equal cost and its
// warps take tiles from it in turn.  Lane r owns row 32t + r and accumulates
// it in a register; per-row loads and stores are coalesced.  One lane
// streams the tile's descriptors into a double-buffered shared-memory stage
// with TMA bulk copies (cp.async.bulk, completion on an mbarrier), one
// segment (or the next tile's first segment) ahead, while the warp reads
// the current segment by broadcast and gathers w.  Only w is kept between
// iterations (ping-pong): x[v] = w[v] * outdeg[v] (or w[v] for a node
// without out-edges).  Residual
// sum |x'-x|, next D and sum x' are accumulated as exact 64-bit fixed-point
// integers (quantum 2^-60, converted with integer instructions), added per
// block into a triple-buffered accumulator of the job, which every block
// reads after the grid barrier; integer sums do not depend on order, so all
// blocks take the same stopping decision and results are deterministic
// however tiles were scheduled.
// Every wait (grid barrier, mbarrier) is bounded; on expiry the kernel
// records FFG_ERR_TIMEOUT, lets its own copies land, and returns.
#include "ffg_internal.cuh"

namespace ffg {

namespace {

// Warps per block: a single solve runs one block of kWarpsSingle warps per
// SM, so that all warps of an SM share one tile counter (warps of one SM are
// not served equally: with several blocks per SM the youngest block finishes
// last).  A batch runs one job (or one rank of a job) per block at a time, in
// blocks of kWarpsBatch warps (several per SM), kWarpsBatchWide warps (one
// per SM, 128 registers per thread) or kWarpsSingle warps (one per SM).  The
// batch kernel holds each job's pointers in registers, where the single
// kernel reads them from its parameters; at 80 registers per thread that
// spills in the tile loop, so the 16-warp form, which has room for them,
// runs the large jobs of a batch faster than the 24-warp one.
#ifndef FFG_PR_WARPS
#define FFG_PR_WARPS 24
#endif
constexpr int kWarpsSingle = FFG_PR_WARPS;
#ifndef FFG_PR_WARPS64
#define FFG_PR_WARPS64 32
#endif
constexpr int kWarpsSingle64 = FFG_PR_WARPS64;  // single FP64 solves
constexpr int kWarpsBatch = 8;
constexpr int kWarpsBatchWide = 16;
constexpr int kMaxBlocks = 4096;
// a block's barrier targets (phase * blocks, phase <= max_iter + 3) fit the
// 32-bit arrival counter
static_assert((uint64_t(FFG_MAX_ITER) + 3) * kMaxBlocks < (uint64_t(1) << 32),
              "barrier targets fit 32 bits");
constexpr uint64_t kTimeoutNs = 2000000000ULL;
#ifndef FFG_PR_SEG
#define FFG_PR_SEG 128
#endif
#ifndef FFG_PR_UNROLL
#define FFG_PR_UNROLL 8
#endif
#ifndef FFG_PR_STEP32
#define FFG_PR_STEP32 16
#endif
#ifndef FFG_PR_MINBLOCKS
#define FFG_PR_MINBLOCKS 3
#endif
constexpr int kSegD = FFG_PR_SEG;       // descriptors per TMA segment
constexpr int kU = FFG_PR_UNROLL;       // descriptor padding unit
static_assert(kU % 2 == 0 && kSegD % kU == 0 && kU <= 32, "descriptor padding");
// The FP64 form whose w is stored as 128-bit fixed point (see Rows below);
// `double` is the FP64 form with w stored as double.
struct F64x {};
// graphs up to this many nodes keep the 16-byte fixed-point w (two buffers
// of 16 N bytes stay well inside L2 next to the descriptors); larger ones
// store w as double and convert each gathered value instead
constexpr int64_t kFxMaxNodes = int64_t(1) << 21;

// Descriptors per step of the gather loop (gathers in flight per lane): a
// multiple of kU; the remainder of a segment is done in steps of kU.  The
// FP64 forms take 8 (their wider gathers need the registers).
template <typename T> struct Step { static constexpr int value = 8; };
template <> struct Step<float> { static constexpr int value = FFG_PR_STEP32; };
static_assert(FFG_PR_STEP32 % kU == 0 && kSegD % FFG_PR_STEP32 == 0 && 8 % kU == 0,
              "gather step");
constexpr int kLayoutThreads = 64;
constexpr int64_t kRowCost = 20;        // per-row cost in in-edge units (batch plan)
constexpr int64_t kTileCost = 19;       // per-tile cost in descriptor units (block split)

// Control block of one job (zeroed by the host before each run).  acc[b]
// holds the fixed-point sums (residual, dangling mass, sum of x) of the
// phases p with (p - 1) % 3 == b: blocks add theirs before the phase's
// barrier, everyone reads them after it, and rank 0 clears the next buffer
// during the phase (its last readers passed the previous barrier).
struct PrCtl {
    unsigned int barrier;
    int status;
    int iters;
    int converged;
    double residual;
    int nblocks;
    int pad;
    unsigned long long acc[3][4];
    unsigned long long busy_ns;  // sum over the job's blocks of their time on it
};

struct PrWs {
    PrCtl *ctl;
    void *w0, *w1;
    double *rinv;         // FP64: 1 / outdeg per row
    uint2 *desc;          // tile descriptors (off, mask)
    int32_t *cnt;         // per tile: descriptors, padded to a multiple of kU
    uint2 *tinfo;         // per tile: (first descriptor / kU, cnt)
    int64_t *tpre;        // exclusive prefix sums of cnt (ntiles + 1)
    int64_t *scan;        // scan scratch (tiles)
    int32_t *perm;        // row of each tile slot
    int32_t *aflag;       // per row: has in-edges
    int64_t *apre;        // exclusive prefix sums of aflag (n + 1)
    int64_t *ascan;       // scan scratch (rows)
    size_t bytes;
};

// first descriptor of tile t, whose first in-edge is e0: every tile has room
// for one descriptor per in-edge plus its padding, and starts 64-byte aligned
__host__ __device__ __forceinline__ int64_t desc_begin(int64_t e0, int64_t t) {
    return (e0 + kU - 1) / kU * kU + 2 * kU * t;
}
inline int64_t desc_capacity(int64_t n, int64_t e) { return e + 2 * kU * ((n + 31) / 32 + 1); }
// tile descriptors are addressed in units of kU by 32-bit indices
inline bool desc_fits(int64_t n, int64_t e) { return desc_capacity(n, e) / kU < (int64_t(1) << 32); }

// w is stored in 4 bytes (FP32) or 16 (FP64 fixed point); FP64 also keeps
// 1 / outdeg per row
inline size_t w_bytes(ffg_prec prec) { return prec == FFG_F32 ? 4 : 16; }

PrWs carve(void *base, int64_t n, int64_t e, ffg_prec prec) {
    Carver c(base);
    PrWs w;
    w.ctl = c.take<PrCtl>(1);
    w.w0 = c.take<char>(size_t(n) * w_bytes(prec));
    w.w1 = c.take<char>(size_t(n) * w_bytes(prec));
    w.rinv = prec == FFG_F64 ? c.take<double>(size_t(n)) : nullptr;
    w.desc = c.take<uint2>(size_t(desc_capacity(n, e)));
    w.cnt = c.take<int32_t>(size_t((n + 31) / 32));
    w.tinfo = c.take<uint2>(size_t((n + 31) / 32));
    w.tpre = c.take<int64_t>(size_t((n + 31) / 32) + 1);
    w.scan = c.take<int64_t>(size_t(scan_scratch_elems((n + 31) / 32)));
    w.perm = c.take<int32_t>(size_t(n));
    w.aflag = c.take<int32_t>(size_t(n));
    w.apre = c.take<int64_t>(size_t(n) + 1);
    w.ascan = c.take<int64_t>(size_t(scan_scratch_elems(n)));
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

// Liveness of the PageRank kernels of this context: every block adds one
// each time it publishes a phase's sums.  A bounded wait restarts its clock
// whenever the count moves, so a group may wait for ranks that are busy with
// an earlier job for as long as that job takes, and gives up only after
// kTimeoutNs in which no block anywhere made progress.
__device__ unsigned int g_heartbeat;
__device__ __forceinline__ void beat() {
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], 1;" ::"l"(&g_heartbeat) : "memory");
}
__device__ __forceinline__ unsigned heartbeat() { return *(volatile unsigned *)&g_heartbeat; }

// Barrier over the `group` blocks of one job (all co-resident: cooperative
// launch).  Bounded: gives up after kTimeoutNs (or 2^24 polls) without
// progress anywhere (see beat), records FFG_ERR_TIMEOUT.  Returns false
// (uniformly for the whole block) if the run must stop.
__device__ bool group_barrier(PrCtl *ctl, unsigned target, int group) {
    __shared__ int s_ok;
    __syncthreads();
    if (group == 1) return true;  // a one-block group only needs the block barrier
    if (threadIdx.x == 0) {
        // release: this block's writes (ordered before by the block barrier)
        // become visible to every block that acquires the count
        red_release_add(&ctl->barrier, 1u);
        uint64_t t0 = global_ns();
        unsigned ns = 0, hb = heartbeat();
        int ok = 1;
        for (uint32_t polls = 0; ld_acquire(&ctl->barrier) < target; ++polls) {
            if ((polls & 15) == 15) {
                if (*(volatile int *)&ctl->status != 0) { ok = 0; break; }
                const unsigned h = heartbeat();
                if (h != hb) {  // some block progressed: wait on
                    hb = h;
                    t0 = global_ns();
                    polls = 0;
                }
            }
            if (polls > (1u << 24) || global_ns() - t0 > kTimeoutNs) {
                atomicCAS(&ctl->status, 0, (int)FFG_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            if (polls > 64) {  // spin briefly, then back off
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

// The same barrier in two halves, for the iteration loop: thread 0 arrives
// as soon as the block's sums are published (its block barrier has ordered
// the block's writes before), the block does work that needs no other block
// (loads for its next tiles), and only then waits.
__device__ __forceinline__ void group_arrive(PrCtl *ctl, int group) {
    if (threadIdx.x == 0 && group > 1) red_release_add(&ctl->barrier, 1u);
}
__device__ bool group_wait(PrCtl *ctl, unsigned target, int group) {
    __shared__ int s_ok;
    if (group == 1) {
        __syncthreads();
        return true;
    }
    if (threadIdx.x == 0) {
        uint64_t t0 = global_ns();
        unsigned ns = 0, hb = heartbeat();
        int ok = 1;
        for (uint32_t polls = 0; ld_acquire(&ctl->barrier) < target; ++polls) {
            if ((polls & 15) == 15) {
                if (*(volatile int *)&ctl->status != 0) { ok = 0; break; }
                const unsigned h = heartbeat();
                if (h != hb) {  // some block progressed: wait on
                    hb = h;
                    t0 = global_ns();
                    polls = 0;
                }
            }
            if (polls > (1u << 24) || global_ns() - t0 > kTimeoutNs) {
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

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------

// The residual, the dangling mass and the sum of x are accumulated as 64-bit
// fixed-point integers with quantum 2^-60 (all three are sums of
// non-negative values below 8).  Integer sums are exact and independent of
// order, so they are deterministic however tiles are scheduled.  Each
// conversion truncates, floor(x * 2^60), without conversions to 64-bit
// integers (those, like FP64 arithmetic, run on a narrow pipe on this
// part): an FP32 value splits into floor(x * 2^28) and the rest of x * 2^28
// times 2^32, both exact in FP32 and converted to 32 bits (the same integer
// as shifting the significand into place, for every float below 4: checked
// exhaustively on the host); an FP64 value has its significand shifted into
// place with integer instructions.
constexpr double kFix = 1152921504606846976.0;  // 2^60
constexpr long long kFixSat = 1LL << 62;        // stands for values >= 4 (never reached)
#ifndef FFG_PR_FIXCONV
#define FFG_PR_FIXCONV 1
#endif
__device__ __forceinline__ long long to_fix(float x) {  // x >= 0
#if FFG_PR_FIXCONV
    if (!(x < 4.0f)) return kFixSat;
    const float y = __fmul_rn(x, 268435456.0f);  // x * 2^28, exact
    const float h = floorf(y);
    const uint32_t hi = static_cast<uint32_t>(h);  // < 2^30
    const uint32_t lo = static_cast<uint32_t>(__fmul_rn(__fsub_rn(y, h), 4294967296.0f));
    return static_cast<long long>((static_cast<unsigned long long>(hi) << 32) | lo);
#else
    const uint32_t b = __float_as_uint(x);
    if (b < 0x00800000u) return 0;                    // zero or below 2^-126
    const int e = static_cast<int>(b >> 23) - 90;     // x * 2^60 = m * 2^e
    const unsigned long long m = (b & 0x7fffffu) | 0x800000u;
    if (e >= 39) return kFixSat;
    return e >= 0 ? static_cast<long long>(m << e) : (e > -24 ? static_cast<long long>(m >> -e) : 0);
#endif
}
__device__ __forceinline__ long long to_fix(double x) {  // x >= 0
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    if (b < 0x0010000000000000ULL) return 0;            // zero or subnormal
    const int e = static_cast<int>(b >> 52) - 1015;     // x * 2^60 = m * 2^e
    const unsigned long long m = (b & 0xfffffffffffffULL) | 0x10000000000000ULL;
    if (e >= 10) return kFixSat;
    return e >= 0 ? static_cast<long long>(m << e) : (e > -53 ? static_cast<long long>(m >> -e) : 0);
}

struct Fix3 {
    long long r = 0, d = 0, s = 0;
};

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block sums of the three accumulators; valid in thread 0
template <int W>
__device__ __forceinline__ Fix3 block_sum_fix(Fix3 v) {
    __shared__ long long red[3][W];
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
        for (int k = 0; k < W; ++k) {
            t.r += red[0][k];
            t.d += red[1][k];
            t.s += red[2][k];
        }
    return t;
}

// thread 0: add the block's sums into buffer `buf`; rank 0 also clears the
// buffer of the next phase
__device__ __forceinline__ void publish(PrCtl *ctl, int buf, const Fix3 &b, int rank) {
    beat();
    if (b.r) atomicAdd(&ctl->acc[buf][0], static_cast<unsigned long long>(b.r));
    if (b.d) atomicAdd(&ctl->acc[buf][1], static_cast<unsigned long long>(b.d));
    if (b.s) atomicAdd(&ctl->acc[buf][2], static_cast<unsigned long long>(b.s));
    if (rank == 0) {
        unsigned long long *nx = ctl->acc[buf == 2 ? 0 : buf + 1];
        nx[0] = 0;
        nx[1] = 0;
        nx[2] = 0;
    }
}

// ---------------------------------------------------------------------------
// descriptor layout of the in-edges (built once per graph)
// ---------------------------------------------------------------------------
// Tiles are made of slots: the rows with in-edges first, ascending, then
// the rows without (their sum is empty: x' = the teleport term), so that no
// lane of a tile with descriptors idles on an empty row.  perm[slot] = row.
// apre holds the exclusive prefix sums of (in-degree > 0) over the rows,
// from any base apre[0]; the number of rows with in-edges is apre[n] -
// apre[0].
__device__ __forceinline__ void active_flag(const int64_t *__restrict__ in_ptr, int64_t v,
                                            int32_t *__restrict__ flag) {
    flag[v] = in_ptr[v + 1] > in_ptr[v] ? 1 : 0;
}
__device__ __forceinline__ void place_row(const int64_t *__restrict__ apre, int64_t n, int64_t v,
                                          int32_t *__restrict__ perm) {
    const int64_t base = apre[0];
    const int64_t p = apre[v] - base;
    const bool act = apre[v + 1] > apre[v];
    perm[act ? p : apre[n] - base + v - p] = static_cast<int32_t>(v);
}

__global__ void k_active_flags(const int64_t *__restrict__ in_ptr, int64_t n,
                               int32_t *__restrict__ flag) {
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
         v += int64_t(gridDim.x) * blockDim.x)
        active_flag(in_ptr, v, flag);
}
__global__ void k_perm(const int64_t *__restrict__ apre, int64_t n, int32_t *__restrict__ perm) {
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
         v += int64_t(gridDim.x) * blockDim.x)
        place_row(apre, n, v, perm);
}

// One tile (one warp): merge the 32 ascending in-lists of its slots' rows by
// offset src - row; each distinct offset becomes one descriptor whose mask
// holds the lanes that have it.  Offsets fit int32 (n < 2^31); INT32_MAX
// marks an exhausted list.  The in-edges of the slots before this tile
// number in_ptr[perm[32t]] when that row has in-edges (all earlier slots
// hold smaller rows with in-edges), else all of them (e).
// A range of rows of a larger graph is laid out the same way: in_ptr then
// starts at the range's first row (its first in-edge is number ebase), e is
// the range's end, and offsets are taken from the global row (row0 + local
// row), so that they index the w of every row.
__device__ void layout_tile(const int64_t *__restrict__ in_ptr,
                            const int32_t *__restrict__ in_idx,
                            const int32_t *__restrict__ perm, int64_t n, int64_t e, int64_t ebase,
                            int64_t row0, uint2 *__restrict__ desc, int32_t *__restrict__ cnt,
                            uint2 *__restrict__ tinfo, int64_t t, int lane) {
    const int64_t slot = (t << 5) + lane;
    int32_t vi = 0;
    int64_t cur = 0, end = 0;
    if (slot < n) {
        vi = perm[slot];
        cur = in_ptr[vi];
        end = in_ptr[vi + 1];
    }
    const int64_t c0 = __shfl_sync(0xffffffffu, cur, 0);  // slot 32t exists
    const int64_t z0 = __shfl_sync(0xffffffffu, end, 0);
    const int64_t dbeg = desc_begin((z0 > c0 ? c0 : e) - ebase, t);
    uint2 *out = desc + dbeg;
    const int32_t row = static_cast<int32_t>(row0 + vi);  // global row, < 2^31
    int32_t head = cur < end ? __ldg(in_idx + cur) - row : INT32_MAX;
    int k = 0;
#ifdef FFG_CHECKED
    // the tile's room: one descriptor per in-edge plus the padding
    int64_t room = end - cur;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) room += __shfl_xor_sync(0xffffffffu, room, o);
    room += kU;
#endif
    while (true) {
        const int32_t m = __reduce_min_sync(0xffffffffu, head);
        if (m == INT32_MAX) break;
        const bool hit = head == m;
        const unsigned mask = __ballot_sync(0xffffffffu, hit);
        if (lane == 0 && FFG_CHECK(k < room, 102)) out[k] = make_uint2(static_cast<uint32_t>(m), mask);
        ++k;
        if (hit) {
            ++cur;
            head = cur < end ? __ldg(in_idx + cur) - row : INT32_MAX;
        }
    }
    const int padded = (k + kU - 1) / kU * kU;
    if (k + lane < padded && FFG_CHECK(k + lane < room, 102)) out[k + lane] = make_uint2(0u, 0u);
    if (lane == 0) {
        cnt[t] = padded;
        tinfo[t] = make_uint2(static_cast<uint32_t>(dbeg / kU), static_cast<uint32_t>(padded));
    }
}

__global__ void __launch_bounds__(kLayoutThreads) k_pr_layout(
    const int64_t *__restrict__ in_ptr, const int32_t *__restrict__ in_idx,
    const int32_t *__restrict__ perm, int64_t n, int64_t e, int64_t ebase, int64_t row0,
    uint2 *__restrict__ desc, int32_t *__restrict__ cnt, uint2 *__restrict__ tinfo) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t ntiles = (n + 31) >> 5;
    const int64_t step = int64_t(gridDim.x) * (kLayoutThreads / 32);
    for (int64_t t = int64_t(blockIdx.x) * (kLayoutThreads / 32) + warp; t < ntiles; t += step)
        layout_tile(in_ptr, in_idx, perm, n, e, ebase, row0, desc, cnt, tinfo, t, lane);
}

// ---------------------------------------------------------------------------
// per-iteration tile work
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// per-precision storage of w and the update of one row
// ---------------------------------------------------------------------------
// FP32: w is a float; in-sums, x' and w' are FP32.
// FP64: w is stored exactly as a 128-bit fixed-point integer (Fx, quantum
// 2^-120; w < 2 fits, and a w below 2^-120 would lose at most one quantum),
// so a row's in-sum is exact, formed by integer additions, and rounded to
// double once.  x' = alpha*S + c and w' = x' * (1/outdeg) are the only FP64
// operations per row; the residual and the dangling mass are taken from the
// fixed-point values.  A warp-wide FP64 add occupies the FP64 units of an SM
// for 16 cycles on this part, so the integer form is the fast one as well
// as the exact one.
struct __align__(16) Fx {
    unsigned long long lo, hi;  // value / 2^-120
};

__device__ __forceinline__ Fx fx_add(Fx a, Fx b) {
    Fx r;
    r.lo = a.lo + b.lo;
    r.hi = a.hi + b.hi + (r.lo < b.lo ? 1ULL : 0ULL);
    return r;
}

// w >= 0 (truncated to the quantum)
__device__ __forceinline__ Fx fx_of(double w) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(w));
    const int e = static_cast<int>(b >> 52);
    const unsigned long long m = (b & 0xfffffffffffffULL) | (e ? 0x10000000000000ULL : 0ULL);
    const int sh = e - 955;  // w / 2^-120 = m * 2^sh, sh < 75 for w < 2
    Fx r;
    if (sh >= 64) {
        r.lo = 0;
        r.hi = m << (sh - 64);
    } else if (sh > 0) {
        r.lo = m << sh;
        r.hi = m >> (64 - sh);
    } else if (sh > -64) {
        r.lo = m >> -sh;
        r.hi = 0;
    } else {
        r.lo = r.hi = 0;
    }
    return r;
}

// to double, rounded to nearest even, with integer instructions
__device__ __forceinline__ double dbl_of(Fx a) {
    if ((a.hi | a.lo) == 0) return 0.0;
    const int lz = a.hi ? __clzll(static_cast<long long>(a.hi))
                        : 64 + __clzll(static_cast<long long>(a.lo));
    unsigned long long h;  // the value shifted so that its leading one is bit 127
    bool tail;             // a one below the 64 bits of h
    if (lz >= 64) {
        h = a.lo << (lz - 64);
        tail = false;
    } else if (lz > 0) {
        h = (a.hi << lz) | (a.lo >> (64 - lz));
        tail = (a.lo << lz) != 0;
    } else {
        h = a.hi;
        tail = a.lo != 0;
    }
    unsigned long long mant = h >> 11;  // 53 bits with the leading one
    const bool round = (h >> 10) & 1ULL;
    const bool sticky = (h & 0x3ffULL) != 0 || tail;
    long long e = 127 - lz - 120 + 1023;  // biased exponent of the leading one
    if (round && (sticky || (mant & 1ULL))) {
        ++mant;
        if (mant >> 53) {
            mant >>= 1;
            ++e;
        }
    }
    return __longlong_as_double((e << 52) | static_cast<long long>(mant & 0xfffffffffffffULL));
}

// a * k for an out-degree k
__device__ __forceinline__ Fx fx_mul(Fx a, uint32_t k) {
    Fx r;
    r.lo = a.lo * k;
    r.hi = a.hi * k + __umul64hi(a.lo, k);
    return r;
}

__device__ __forceinline__ Fx fx_absdiff(Fx a, Fx b) {
    const bool ge = a.hi > b.hi || (a.hi == b.hi && a.lo >= b.lo);
    const Fx x = ge ? a : b, y = ge ? b : a;
    Fx r;
    r.lo = x.lo - y.lo;
    r.hi = x.hi - y.hi - (x.lo < y.lo ? 1ULL : 0ULL);
    return r;
}

// the 2^-60 fixed-point form of the reductions (value < 8)
__device__ __forceinline__ long long fix60(Fx a) {
    return static_cast<long long>((a.hi << 4) | (a.lo >> 60));
}

template <typename T>
struct Rows;

template <>
struct Rows<float> {
    using Real = float;
    using W = float;
    struct Extra {};
    __device__ static W init(double x0, int od) { return static_cast<float>(od ? x0 / od : x0); }
    __device__ static void store_rinv(double *, int64_t, int) {}
    __device__ static double x_of(W w, int od) {
        return od ? static_cast<double>(w) * od : static_cast<double>(w);
    }
    __device__ static long long fix_x(W w, int od) { return to_fix(x_of(w, od)); }
    __device__ static void load_extra(Extra &, const double *, int) {}
    // x' = alpha*s + c from the row's in-sum; w' = x'/outdeg as x' times the
    // correctly rounded reciprocal (two roundings, no division sequence)
    __device__ static void update(float s, float a, float c, int od, W wold, const Extra &,
                                  W *dst, Fix3 &f) {
        const float xo = od ? wold * static_cast<float>(od) : wold;
        const float xn = a * s + c;
        f.r += to_fix(xn > xo ? xn - xo : xo - xn);
        if (od == 0) f.d += to_fix(xn);
        *dst = od ? xn * __frcp_rn(static_cast<float>(od)) : xn;
    }
};

template <>
struct Rows<double> {
    using Real = double;
    using W = double;
    struct Extra {
        double rinv;  // 1 / outdeg (1 without out-edges)
    };
    __device__ static W init(double x0, int od) { return od ? x0 / od : x0; }
    __device__ static double x_of(W w, int od) { return od ? w * od : w; }
    __device__ static long long fix_x(W w, int od) { return to_fix(x_of(w, od)); }
    __device__ static void store_rinv(double *rinv, int64_t v, int od) {
        rinv[v] = od ? 1.0 / od : 1.0;
    }
    __device__ static void load_extra(Extra &e, const double *rinv, int v) {
        e.rinv = v >= 0 ? rinv[v] : 1.0;  // written by the prologue: a plain load
    }
    __device__ static void update(double s, double a, double c, int od, W wold, const Extra &e,
                                  W *dst, Fix3 &f) {
        const double xo = od ? wold * od : wold;
        const double xn = fma(a, s, c);
        f.r += to_fix(xn > xo ? xn - xo : xo - xn);
        if (od == 0) f.d += to_fix(xn);
        *dst = od ? xn * e.rinv : xn;
    }
};

template <>
struct Rows<F64x> {
    using Real = double;
    using W = Fx;
    struct Extra {
        double rinv;  // 1 / outdeg (1 without out-edges)
    };
    __device__ static W init(double x0, int od) { return fx_of(od ? x0 / od : x0); }
    __device__ static double x_of(W w, int od) {
        return dbl_of(od ? fx_mul(w, static_cast<uint32_t>(od)) : w);
    }
    __device__ static long long fix_x(W w, int od) {
        return fix60(od ? fx_mul(w, static_cast<uint32_t>(od)) : w);
    }
    __device__ static void store_rinv(double *rinv, int64_t v, int od) {
        rinv[v] = od ? 1.0 / od : 1.0;
    }
    __device__ static void load_extra(Extra &e, const double *rinv, int v) {
        e.rinv = v >= 0 ? rinv[v] : 1.0;  // written by the prologue: a plain load
    }
    __device__ static void update(double s, double a, double c, int od, W wold, const Extra &e,
                                  W *dst, Fix3 &f) {
        const double xn = fma(a, s, c);
        const Fx xf = fx_of(xn);
        const Fx xo = od ? fx_mul(wold, static_cast<uint32_t>(od)) : wold;
        f.r += fix60(fx_absdiff(xf, xo));
        if (od == 0) f.d += fix60(xf);
        *dst = od ? fx_of(xn * e.rinv) : xf;
    }
};

template <typename T>
struct TileInfo {
    uint32_t d8;                        // first descriptor / kU
    int cnt;                            // descriptors (multiple of kU)
    int32_t v;                          // this lane's row (-1 past the last slot)
    int32_t od;                         // its out-degree
    typename Rows<T>::W wv;             // its w
    typename Rows<T>::Extra ex;         // its per-precision row data
};

// A tile's info loads in two steps, a tile apart, so that no load waits on
// the one before it: its head (descriptor range and this lane's row), then
// the row's data (out-degree and w), which need the row.
template <typename T>
__device__ __forceinline__ TileInfo<T> load_head(int t, int n, const uint2 *__restrict__ tinfo,
                                                 const int32_t *__restrict__ perm, int lane) {
    TileInfo<T> ti;
    const int slot = (t << 5) + lane;  // n < 2^31
    const uint2 h = __ldg(tinfo + t);
    ti.d8 = h.x;
    ti.cnt = static_cast<int>(h.y);
    ti.v = slot < n ? __ldg(perm + slot) : -1;
    ti.od = 0;
    ti.wv = typename Rows<T>::W{};
    ti.ex = typename Rows<T>::Extra{};
    return ti;
}
template <typename T>
__device__ __forceinline__ void load_row(TileInfo<T> &ti, const int32_t *__restrict__ outdeg,
                                         const typename Rows<T>::W *wc, const double *rinv) {
    ti.od = ti.v >= 0 ? __ldg(outdeg + ti.v) : 0;
    ti.wv = ti.v >= 0 ? wc[ti.v] : typename Rows<T>::W{};
    Rows<T>::load_extra(ti.ex, rinv, ti.v);
}

// Per-warp TMA stream of descriptor segments into a two-buffer stage.
// `pending` has bit b set while a copy into buffer b is outstanding.
struct Stream {
    uint2 *stage;      // [2][kSegD]
    uint64_t *bar;     // [2]
    uint32_t phase;    // bit b = parity of the next completion on buffer b
    uint32_t pending;  // bit b = a copy into buffer b is outstanding
    int buf;           // buffer of the segment to process next
    bool issued;       // the segment for `buf` has been issued
    // copy `count` descriptors (a multiple of kU: 64-byte multiples, 64-byte
    // aligned source) into buffer b
    __device__ __forceinline__ void issue(const uint2 *src, int count, int b, int lane) {
        if (lane == 0)
            tma_load(stage + b * kSegD, src, static_cast<uint32_t>(count) * 8u, bar + b);
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

// The lane has an in-edge at offset `off` of descriptor mask `mask`; in a
// bounds-checked build the gather must also stay inside w: gb = [lo, hi) of
// the offsets that do, for this lane's row.
__device__ __forceinline__ bool take(uint32_t mask, uint32_t bit, uint32_t off, int2 gb) {
    return (mask & bit) &&
           FFG_CHECK(static_cast<int32_t>(off) >= gb.x && static_cast<int32_t>(off) < gb.y, 101);
}

// N descriptors (q: N/2 pairs, the same for every lane): the sum of this
// lane's gathers, added pairwise.
template <typename T, int N>
__device__ __forceinline__ T gather_step(const uint4 *q, const T *wrow, uint32_t bit, int2 gb) {
    T v[N];
#pragma unroll
    for (int j = 0; j < N / 2; ++j) {
        const uint4 d = q[j];  // two descriptors, read by broadcast
        v[2 * j] = take(d.y, bit, d.x, gb) ? wrow[static_cast<int32_t>(d.x)] : T(0);
        v[2 * j + 1] = take(d.w, bit, d.z, gb) ? wrow[static_cast<int32_t>(d.z)] : T(0);
    }
#pragma unroll
    for (int h = N / 2; h > 0; h >>= 1)  // depth log2(N)
#pragma unroll
        for (int j = 0; j < h; ++j) v[j] += v[j + h];
    return v[0];
}

// Per-lane accumulator of a row's in-sum: FP32 pairwise partial sums added
// in order; FP64 exact 128-bit integer sums (of stored fixed-point values, or
// of doubles converted as they are gathered).
template <typename T>
struct Accum;

template <>
struct Accum<float> {
    float s = 0.f;
    template <int N>
    __device__ __forceinline__ void step(const uint4 *q, const float *wrow, uint32_t bit, int2 gb) {
        s += gather_step<float, N>(q, wrow, bit, gb);
    }
    __device__ __forceinline__ float value() const { return s; }
};

template <>
struct Accum<double> {
    Fx s{0ULL, 0ULL};
    template <int N>
    __device__ __forceinline__ void step(const uint4 *q, const double *wrow, uint32_t bit,
                                         int2 gb) {
        double v[N];
#pragma unroll
        for (int j = 0; j < N / 2; ++j) {
            const uint4 d = q[j];
            v[2 * j] = take(d.y, bit, d.x, gb) ? wrow[static_cast<int32_t>(d.x)] : 0.0;
            v[2 * j + 1] = take(d.w, bit, d.z, gb) ? wrow[static_cast<int32_t>(d.z)] : 0.0;
        }
#pragma unroll
        for (int j = 0; j < N; ++j) s = fx_add(s, fx_of(v[j]));
    }
    __device__ __forceinline__ double value() const { return dbl_of(s); }
};

template <>
struct Accum<F64x> {
    Fx s{0ULL, 0ULL};
    template <int N>
    __device__ __forceinline__ void step(const uint4 *q, const Fx *wrow, uint32_t bit, int2 gb) {
        Fx v[N];
#pragma unroll
        for (int j = 0; j < N / 2; ++j) {
            const uint4 d = q[j];
            v[2 * j] = take(d.y, bit, d.x, gb) ? wrow[static_cast<int32_t>(d.x)] : Fx{0ULL, 0ULL};
            v[2 * j + 1] = take(d.w, bit, d.z, gb) ? wrow[static_cast<int32_t>(d.z)]
                                                   : Fx{0ULL, 0ULL};
        }
#pragma unroll
        for (int j = 0; j < N; ++j) s = fx_add(s, v[j]);
    }
    __device__ __forceinline__ double value() const { return dbl_of(s); }
};

// Sum over the in-edges of this lane's row (wrow = w + row): the tile's
// `cnt` descriptors (from dcur) stream in segments of kSegD; the segment
// after the current one (or the first segment of the next tile: ncnt
// descriptors from dnxt, when next_any) is copied while the current one is
// gathered.
template <typename T>
__device__ __forceinline__ bool tile_sum(const uint2 *dcur, int cnt, const uint2 *dnxt, int ncnt,
                                         bool next_any, Stream &st,
                                         const typename Rows<T>::W *wrow, uint32_t bit, int2 gb,
                                         int lane, typename Rows<T>::Real &sum) {
    const int nseg = (cnt + kSegD - 1) / kSegD;
    Accum<T> acc;
    for (int sg = 0; sg < nseg; ++sg) {
        const int c0 = sg * kSegD;
        const int m = cnt - c0 < kSegD ? cnt - c0 : kSegD;
        if (!st.issued) st.issue(dcur + c0, m, st.buf, lane);
        if (sg + 1 < nseg) {
            const int c1 = c0 + kSegD;
            st.issue(dcur + c1, cnt - c1 < kSegD ? cnt - c1 : kSegD, st.buf ^ 1, lane);
            st.issued = true;
        } else if (next_any) {
            st.issue(dnxt, ncnt < kSegD ? ncnt : kSegD, st.buf ^ 1, lane);
            st.issued = true;
        } else {
            st.issued = false;
        }
        if (!st.wait(st.buf)) return false;
        const uint4 *q = reinterpret_cast<const uint4 *>(st.stage + st.buf * kSegD);
        constexpr int kS = Step<T>::value;
        int k = 0;
        for (; k + kS <= m; k += kS) acc.template step<kS>(q + (k >> 1), wrow, bit, gb);
        if (kS > kU)
            for (; k < m; k += kU) acc.template step<kU>(q + (k >> 1), wrow, bit, gb);
        st.buf ^= 1;
    }
    if (nseg == 0 && !st.issued && next_any) {
        st.issue(dnxt, ncnt < kSegD ? ncnt : kSegD, st.buf, lane);
        st.issued = true;
    }
    sum = acc.value();
    return true;
}

// tile_sum for two tiles of one layout
template <typename T>
__device__ __forceinline__ bool tile_sum(const uint2 *__restrict__ desc, const TileInfo<T> &cur,
                                         const TileInfo<T> &nxt, bool has_next, Stream &st,
                                         const typename Rows<T>::W *wrow, uint32_t bit, int2 gb,
                                         int lane, typename Rows<T>::Real &sum) {
    return tile_sum<T>(desc + size_t(cur.d8) * kU, cur.cnt, desc + size_t(nxt.d8) * kU, nxt.cnt,
                       has_next && nxt.cnt > 0, st, wrow, bit, gb, lane, sum);
}

// the offsets whose gather stays inside w (n rows) for row v (bounds checks)
__device__ __forceinline__ int2 gather_bounds(int64_t v, int64_t n) {
    return v < 0 ? make_int2(0, 0)
                 : make_int2(static_cast<int>(-v), static_cast<int>(n - v));
}

// First tile of part w when the tiles are split into nw contiguous ranges of
// about equal cost; a tile costs its descriptors plus kTileCost (the time
// per tile is close to linear in these two).  tpre: prefix sums of the
// descriptor counts (any base).
__device__ __forceinline__ int64_t tile_split(const int64_t *__restrict__ tpre, int64_t ntiles,
                                              int64_t w, int64_t nw) {
    if (w <= 0) return 0;
    if (w >= nw) return ntiles;
    const int64_t base = __ldg(tpre);
    const int64_t total = __ldg(tpre + ntiles) - base + kTileCost * ntiles;
    const int64_t target = total / nw * w + (total % nw) * w / nw;
    int64_t lo = 0, hi = ntiles;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(tpre + mid) - base + kTileCost * mid >= target) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

template <int W>
constexpr size_t pr_smem_bytes() {
    return size_t(W) * (2 * kSegD * sizeof(uint2) + 16);
}

// One PageRank job: a graph, its layout, its buffers and its parameters.
// `group` blocks work on it together (ranks 0..group-1), synchronised by the
// job's own bounded barrier in `ctl`.
struct JobDev {
    const int32_t *outdeg;
    const uint2 *desc;
    const uint2 *tinfo;
    const int32_t *perm;
    double *rinv;  // FP64: 1 / outdeg per row, written by the prologue
    const int64_t *tpre;
    const int64_t *apre;  // rows with in-edges: apre[n] - apre[0]
    void *ranks, *w0, *w1;
    PrCtl *ctl;
    int64_t n;
    double alpha, tol;
    int max_iter, init, group, pad;
};

// Loop state of a job, kept by thread 0 in shared memory: the tile loop
// holds none of it in registers.
struct LoopState {
    double res, prev_res, xs;
    int it, stop, converged, pad;
    uint64_t t0;  // when all ranks had started (for the job's busy time)
};

// the teleport term (alpha * D + 1 - alpha) / n from the fixed-point dangling
// mass D, one rounding per operation (also in the row-range form, so that
// both give the same bits)
__device__ __forceinline__ double teleport(double alpha, unsigned long long d_fix, int64_t n) {
    const double d = static_cast<double>(d_fix) / kFix;
    return __dsub_rn(__dadd_rn(__dmul_rn(alpha, d), 1.0), alpha) / static_cast<double>(n);
}

// thread 0, after the barrier of an iteration: read the job's sums, decide
// whether to stop, and publish the next teleport term
template <typename T>
__device__ __forceinline__ void advance(const JobDev &J, LoopState &ls, const PrCtl *ctl, int buf,
                                        T *s_c, bool count_iter) {
    const double r = static_cast<double>(__ldcg(&ctl->acc[buf][0])) / kFix;
    *s_c = static_cast<T>(teleport(J.alpha, __ldcg(&ctl->acc[buf][1]), J.n));
    if (!count_iter) return;  // the prologue: no iteration yet
    ls.prev_res = ls.res;
    ls.res = r;
    ++ls.it;
    if (r < J.tol) ls.converged = ls.stop = 1;
    else if (sizeof(T) == 4 && r >= ls.prev_res) ls.converged = ls.stop = 1;  // FP32 floor
    else if (ls.it >= J.max_iter) ls.stop = 1;
}

// A group of blocks runs all iterations of one job.  Returns false if the
// block must stop (a bounded wait expired).
template <typename T, int W>
__device__ bool run_job(const JobDev &J, int rank, Stream &st) {
    constexpr int kThreads = 32 * W;
    using R = typename Rows<T>::Real;  // arithmetic type
    const int32_t *__restrict__ outdeg = J.outdeg;
    const uint2 *__restrict__ desc = J.desc;
    const uint2 *__restrict__ tinfo = J.tinfo;
    const int32_t *__restrict__ perm = J.perm;
    const int64_t n = J.n;
    const int nb = J.group;
    using WS = typename Rows<T>::W;
    WS *w0 = static_cast<WS *>(J.w0), *w1 = static_cast<WS *>(J.w1);
    double *rinv = J.rinv;  // 1 / outdeg per row
    PrCtl *ctl = J.ctl;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // Tiles hold the slots of the rows with in-edges (the last one may also
    // hold rows without); the remaining slots, rows whose sum is empty, are
    // done element-wise by every block.  The block's contiguous tile range has
    // about equal cost per block.  Warp w starts with tiles bt0 + w and
    // bt0 + W + w; the rest are taken in turn through a shared counter.
    __shared__ int s_range[3];
    __shared__ unsigned s_next;
    __shared__ LoopState s_ls;
    __shared__ R s_c;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int64_t ntiles = (J.apre[n] - J.apre[0] + 31) >> 5;
        s_range[2] = static_cast<int>(ntiles);
        s_range[0] = static_cast<int>(tile_split(J.tpre, ntiles, rank, nb));
        s_range[1] = static_cast<int>(tile_split(J.tpre, ntiles, rank + 1, nb));
        s_next = static_cast<unsigned>(s_range[0] + 2 * W);
        s_ls.res = __longlong_as_double(0x7ff0000000000000LL);
        s_ls.it = s_ls.stop = s_ls.converged = 0;
    }
    __syncthreads();
    const int bt0 = s_range[0], bt1 = s_range[1];
    const int64_t slot_empty = int64_t(s_range[2]) << 5;  // first slot done element-wise
    const int ni = static_cast<int>(n);

    // prologue: w from the start vector and D_0 (grid-stride)
    {
        const double inv_n = 1.0 / static_cast<double>(n);
        const R *ranks = static_cast<const R *>(J.ranks);
        Fix3 acc0;
        const int64_t stride = int64_t(nb) * kThreads;
        for (int64_t v = int64_t(rank) * kThreads + threadIdx.x; v < n; v += stride) {
            const double x0 = J.init ? static_cast<double>(ranks[v]) : inv_n;
            const int32_t od = __ldg(outdeg + v);
            w0[v] = Rows<T>::init(x0, od);
            Rows<T>::store_rinv(rinv, v, od);
            if (od == 0) acc0.d += to_fix(x0);
        }
        const Fix3 b = block_sum_fix<W>(acc0);
        if (threadIdx.x == 0) publish(ctl, 0, b, rank);
    }
    unsigned phase = 1;
    int buf = 0;
    if (!group_barrier(ctl, phase * nb, nb)) return false;
    if (threadIdx.x == 0) {
        s_ls.t0 = global_ns();
        advance<R>(J, s_ls, ctl, buf, &s_c, false);
    }
    __syncthreads();
    WS *wc = w0, *wn = w1;
    const R a = static_cast<R>(J.alpha);
    int failed = 0;
    const int t0 = bt0 + warp, t1 = bt0 + W + warp;  // this warp's first two tiles
    TileInfo<T> pre0, pre1;  // ... loaded ahead (have_pre)
    bool have_pre = false;
    while (true) {
        const R c = s_c;
        Fix3 facc;
        if (t0 < bt1 && !failed) {
            // cur: tile being summed; nxt: its successor (info loaded one tile
            // ahead, so its first segment can be issued at once); the tile
            // after nxt is taken and its info loaded while cur is summed
            int t = t0, tn = t1;
            TileInfo<T> cur, nxt;
            if (have_pre) {
                cur = pre0;
                nxt = pre1;
            } else {
                cur = load_head<T>(t0, ni, tinfo, perm, lane);
                nxt = load_head<T>(t1 < bt1 ? t1 : t0, ni, tinfo, perm, lane);
                load_row<T>(cur, outdeg, wc, rinv);
            }
            while (true) {
                const bool has_next = tn < bt1;
                int tn2 = bt1;
                if (has_next) {
                    unsigned g = 0;
                    if (lane == 0) g = atomicAdd(&s_next, 1u);
                    tn2 = static_cast<int>(__shfl_sync(0xffffffffu, g, 0));
                }
                load_row<T>(nxt, outdeg, wc, rinv);
                const TileInfo<T> nx2 = load_head<T>(tn2 < bt1 ? tn2 : t, ni, tinfo, perm, lane);
                const int v = cur.v;
                R s = R(0);
                if (!tile_sum<T>(desc, cur, nxt, has_next, st, wc + (v < 0 ? 0 : v), 1u << lane,
                                 gather_bounds(v, n), lane, s)) {
                    failed = 1;
                    break;
                }
                if (v >= 0) Rows<T>::update(s, a, c, cur.od, cur.wv, cur.ex, wn + v, facc);
                if (!has_next) break;
                cur = nxt;
                t = tn;
                nxt = nx2;
                tn = tn2;
            }
        }
        // rows without in-edges: x' = c
        for (int64_t i = slot_empty + int64_t(rank) * kThreads + threadIdx.x; i < n;
             i += int64_t(nb) * kThreads) {
            const int v = __ldg(perm + i);
            const int32_t od = __ldg(outdeg + v);
            typename Rows<T>::Extra ex;
            Rows<T>::load_extra(ex, rinv, v);
            Rows<T>::update(R(0), a, c, od, wc[v], ex, wn + v, facc);
        }
        if (failed == 1) {
            // let this warp's own copies land (bounded), then report
            st.drain();
            if (lane == 0) atomicCAS(&ctl->status, 0, (int)FFG_ERR_TIMEOUT);
            failed = 2;
        }
        const Fix3 b = block_sum_fix<W>(facc);
        // The block's rows of w' are written (block barrier above): publish
        // the sums and arrive at once.
        buf = buf == 2 ? 0 : buf + 1;
        if (threadIdx.x == 0) {
            publish(ctl, buf, b, rank);
            s_next = static_cast<unsigned>(bt0 + 2 * W);  // next iteration's counter
        }
        group_arrive(ctl, nb);
        ++phase;
        // While the others arrive, the next iteration's first two tiles --
        // in this block's range -- load their row data, and the first one
        // its first descriptor segment.  Unused if the solve stops here
        // (drained below).
        have_pre = false;
        if (t0 < bt1 && !failed) {
            pre0 = load_head<T>(t0, ni, tinfo, perm, lane);
            pre1 = load_head<T>(t1 < bt1 ? t1 : t0, ni, tinfo, perm, lane);
            load_row<T>(pre0, outdeg, wn, rinv);
            if (pre0.cnt > 0 && !st.issued) {
                st.issue(desc + size_t(pre0.d8) * kU, pre0.cnt < kSegD ? pre0.cnt : kSegD, st.buf,
                         lane);
                st.issued = true;
            }
            have_pre = true;
        }
        if (!group_wait(ctl, phase * nb, nb)) {
            st.drain();
            st.issued = false;
            return false;
        }
        if (threadIdx.x == 0) advance<R>(J, s_ls, ctl, buf, &s_c, true);
        __syncthreads();
        WS *tmp = wc;
        wc = wn;
        wn = tmp;
        if (s_ls.stop) break;
    }
    if (st.issued) {  // a segment loaded ahead for an iteration that did not run
        st.drain();
        st.issued = false;
    }
    // epilogue: sum x' (one more phase), then x' normalised to sum 1
    const int64_t stride = int64_t(nb) * kThreads;
    {
        Fix3 accs;
        for (int64_t v = int64_t(rank) * kThreads + threadIdx.x; v < n; v += stride) {
            const int32_t od = __ldg(outdeg + v);
            accs.s += Rows<T>::fix_x(wc[v], od);
        }
        const Fix3 b = block_sum_fix<W>(accs);
        buf = buf == 2 ? 0 : buf + 1;
        if (threadIdx.x == 0) publish(ctl, buf, b, rank);
        ++phase;
        if (!group_barrier(ctl, phase * nb, nb)) return false;
        if (threadIdx.x == 0) s_ls.xs = static_cast<double>(__ldcg(&ctl->acc[buf][2])) / kFix;
        __syncthreads();
    }
    const double inv_s = 1.0 / s_ls.xs;
    R *ranks = static_cast<R *>(J.ranks);
    for (int64_t v = int64_t(rank) * kThreads + threadIdx.x; v < n; v += stride) {
        const int32_t od = __ldg(outdeg + v);
        ranks[v] = static_cast<R>(Rows<T>::x_of(wc[v], od) * inv_s);
    }
    if (threadIdx.x == 0) {
        atomicAdd(&ctl->busy_ns, static_cast<unsigned long long>(global_ns() - s_ls.t0));
        if (rank == 0) {
            ctl->iters = s_ls.it;
            ctl->residual = s_ls.res;
            ctl->converged = s_ls.converged;
            ctl->nblocks = nb;
        }
    }
    return failed == 0;
}

// The persistent kernels: k_pagerank runs one solve on the whole grid,
// k_pagerank_batch the plan's items -- (job, rank) pairs -- in one of two
// orders:
// - lists (queue == nullptr): block b runs items [first[b], first[b+1]),
//   its multi-block rank (if any) first, so no two groups wait on each other;
// - claims: the blocks claim the items in order through a counter (`queue`,
//   zero at launch), a job's ranks being consecutive items, and a block runs
//   its item to the end before it claims another.  So at most one group --
//   the last one claimed -- can be short of ranks: every other group has all
//   of its ranks running and completes, and its blocks then claim the
//   missing ranks (a group has at most as many ranks as the grid has
//   blocks).  No group waits forever.
// shared memory: per-warp stages, then mbarriers
template <int W>
__device__ __forceinline__ Stream make_stream(unsigned char *s_dyn) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Stream st;
    st.stage = reinterpret_cast<uint2 *>(s_dyn) + size_t(warp) * 2 * kSegD;
    st.bar = reinterpret_cast<uint64_t *>(s_dyn + size_t(W) * 2 * kSegD * sizeof(uint2)) +
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
    return st;
}

// One solve on the whole grid.
template <typename T, int W>
__global__ void __launch_bounds__(32 * W, W == kWarpsBatch ? FFG_PR_MINBLOCKS : 1)
    k_pagerank(JobDev single) {
    extern __shared__ __align__(128) unsigned char s_dyn[];
    Stream st = make_stream<W>(s_dyn);
    run_job<T, W>(single, blockIdx.x, st);
}

template <typename T, int W>
__global__ void __launch_bounds__(32 * W, W == kWarpsBatch ? FFG_PR_MINBLOCKS : 1)
    k_pagerank_batch(const JobDev *__restrict__ jobs, const int2 *__restrict__ items,
                     const int *__restrict__ first, int *__restrict__ queue, int n_items) {
    extern __shared__ __align__(128) unsigned char s_dyn[];
    Stream st = make_stream<W>(s_dyn);
    if (queue == nullptr) {
        for (int i = first[blockIdx.x]; i < first[blockIdx.x + 1]; ++i) {
            const int2 item = items[i];
            const JobDev J = jobs[item.x];
            if (!run_job<T, W>(J, item.y, st)) return;
        }
        return;
    }
    __shared__ int s_item;
    while (true) {
        __syncthreads();  // every thread has read the previous item
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        const int i = s_item;
        if (i >= n_items) return;
        const int2 item = items[i];
        const JobDev J = jobs[item.x];
        if (!run_job<T, W>(J, item.y, st)) return;
    }
}

// The same with the job table in the kernel's parameters, for batches of at
// most kParamJobs jobs.  A job's pointers are then read from the constant
// bank where they are used, as in k_pagerank, instead of being held in
// registers for the whole job: at 80 registers per thread those spilled in
// the tile loop (the 24-warp kernel ran the 234-space batch 20 % slower).
constexpr int kParamJobs = FFG_PR_PARAM_JOBS;
static_assert(sizeof(JobDev) == 128 && sizeof(JobDev) * kParamJobs ==
                                           sizeof(((ffg_pr_batch *)nullptr)->params),
              "the plan holds the parameter job table");
struct BatchParams {
    const int2 *items;
    const int *first;
    int *queue;
    int n_items, pad;
    JobDev jobs[kParamJobs];
};
static_assert(sizeof(BatchParams) <= 32764, "kernel parameter limit");

template <typename T, int W>
__global__ void __launch_bounds__(32 * W, W == kWarpsBatch ? FFG_PR_MINBLOCKS : 1)
    k_pagerank_batch_p(const __grid_constant__ BatchParams P) {
    extern __shared__ __align__(128) unsigned char s_dyn[];
    Stream st = make_stream<W>(s_dyn);
    if (P.queue == nullptr) {
        for (int i = P.first[blockIdx.x]; i < P.first[blockIdx.x + 1]; ++i) {
            const int2 item = P.items[i];
            if (!run_job<T, W>(P.jobs[item.x], item.y, st)) return;
        }
        return;
    }
    __shared__ int s_item;
    while (true) {
        __syncthreads();  // every thread has read the previous item
        if (threadIdx.x == 0) s_item = atomicAdd(P.queue, 1);
        __syncthreads();
        const int i = s_item;
        if (i >= P.n_items) return;
        const int2 item = P.items[i];
        if (!run_job<T, W>(P.jobs[item.x], item.y, st)) return;
    }
}

// ---------------------------------------------------------------------------
// The sweep schedule: all jobs of a batch advance in lock-step on the whole
// grid.  A phase is one step of every unfinished job -- its prologue, one
// iteration, the sum of its x, or the write of its normalised ranks -- and
// one grid barrier separates phases.  A step's work is cut into units:
// tiles of 32 slots (an iteration's rows with in-edges) and chunks of
// kSweepRows rows (the element-wise work: prologue, rows without in-edges,
// sum, write), numbered over all jobs, job after job.  Block b owns the
// b-th equal share of a phase's units and its warps claim them in order
// through a counter in global memory; a warp whose block's share is used up
// claims units left in the other blocks' shares, so the phase ends when the
// work does, whatever each unit cost.  After the barrier every block reads
// the jobs' fixed-point sums and takes the same decisions (iteration count,
// stop, teleport term, normalisation) in its own shared-memory copy of the
// jobs' states: exact integer sums do not depend on which block added what.
// One iteration of every job costs one barrier, not one per job, and no
// block waits for another job's blocks.
// ---------------------------------------------------------------------------
constexpr int kSweepRows = 256;   // rows of an element-wise unit
constexpr int kSweepClaim = 2;    // units taken per claim from a block's share
enum : int { kSwInit = 0, kSwIter = 1, kSwSum = 2, kSwWrite = 3, kSwDone = 4 };

// one job's state, identical in every block (shared memory)
struct SwJob {
    double res, prev_res, inv_s, c;
    int mode, it, converged, wsel;  // wsel: the w buffer holding the current x
    int ntiles, nempty, nrows, units;  // tiles, chunks of rows without in-edges, chunks of rows
};

struct SweepCtl {
    unsigned int barrier;  // grid barrier arrivals
    int status;            // first failure (FFG_ERR_TIMEOUT), 0 if none
};
struct SweepRange {
    int tag, start, len, pad;  // the phase it belongs to, its units
};

struct SweepArgs {
    const JobDev *jobs;
    SweepCtl *ctl;
    SweepRange *ranges;  // [2][nb], by phase parity
    int *ctr;            // [2][nb]: units claimed from each block's share
    int n_jobs, nb;
};

template <int W>
constexpr size_t sweep_smem_bytes(int n_jobs) {
    return pr_smem_bytes<W>() + size_t(n_jobs) * (sizeof(SwJob) + sizeof(JobDev)) +
           (size_t(n_jobs) + 1) * sizeof(int);
}

// grid barrier over all nb blocks (bounded); false if the run must stop
__device__ bool sweep_barrier(SweepCtl *ctl, unsigned target, int *s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        red_release_add(&ctl->barrier, 1u);
        uint64_t t0 = global_ns();
        unsigned ns = 0, hb = heartbeat();
        int ok = 1;
        for (uint32_t polls = 0; ld_acquire(&ctl->barrier) < target; ++polls) {
            if ((polls & 15) == 15) {
                if (*(volatile int *)&ctl->status != 0) { ok = 0; break; }
                const unsigned h = heartbeat();
                if (h != hb) {  // some block progressed: wait on
                    hb = h;
                    t0 = global_ns();
                    polls = 0;
                }
            }
            if (polls > (1u << 24) || global_ns() - t0 > kTimeoutNs) {
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
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// A unit: its job, kind (0 none, 1 tile, 2 chunk) and index within the step.
struct SwUnit {
    int job, kind, idx;
};

// global unit u -> its job (binary search over the jobs' first units, from
// the job of the previous unit) and its kind
__device__ __forceinline__ SwUnit sweep_unit(int u, const int *spre, const SwJob *sj, int n_jobs,
                                             int hint) {
    SwUnit r;
    if (u < 0) {
        r.job = 0;
        r.kind = 0;
        r.idx = 0;
        return r;
    }
    int j = hint;
    if (!(spre[j] <= u && u < spre[j + 1])) {
        int lo = 0, hi = n_jobs - 1;  // last job whose first unit is <= u
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (spre[mid] <= u) lo = mid;
            else hi = mid - 1;
        }
        j = lo;
    }
    r.job = j;
    r.idx = u - spre[j];
    r.kind = (sj[j].mode == kSwIter && r.idx < sj[j].ntiles) ? 1 : 2;
    return r;
}

// element-wise unit: chunk `idx` of job J in state s (mode INIT, ITER rows
// without in-edges, SUM or WRITE); each lane takes every 32nd row of the
// chunk, four at a time
template <typename T>
__device__ void sweep_chunk(const JobDev &J, const SwJob &s, int idx, Fix3 &f, int lane) {
    using WS = typename Rows<T>::W;
    using R = typename Rows<T>::Real;
    WS *wb[2] = {static_cast<WS *>(J.w0), static_cast<WS *>(J.w1)};
    const int64_t n = J.n;
    constexpr int kI = 4;
    if (s.mode == kSwInit) {
        const double inv_n = 1.0 / static_cast<double>(n);
        const R *ranks = static_cast<const R *>(J.ranks);
        for (int r0 = 0; r0 < kSweepRows; r0 += 32 * kI) {
            int32_t od[kI];
            double x0[kI];
#pragma unroll
            for (int k = 0; k < kI; ++k) {
                const int64_t v = int64_t(idx) * kSweepRows + r0 + 32 * k + lane;
                od[k] = v < n ? __ldg(J.outdeg + v) : 0;
                x0[k] = (v < n && J.init) ? static_cast<double>(ranks[v]) : inv_n;
            }
#pragma unroll
            for (int k = 0; k < kI; ++k) {
                const int64_t v = int64_t(idx) * kSweepRows + r0 + 32 * k + lane;
                if (v >= n) continue;
                wb[0][v] = Rows<T>::init(x0[k], od[k]);
                Rows<T>::store_rinv(J.rinv, v, od[k]);
                if (od[k] == 0) f.d += to_fix(x0[k]);
            }
        }
        return;
    }
    if (s.mode == kSwIter) {  // rows without in-edges: x' = c
        const WS *wc = wb[s.wsel];
        WS *wn = wb[s.wsel ^ 1];
        const R a = static_cast<R>(J.alpha), c = static_cast<R>(s.c);
        const int64_t base = (int64_t(s.ntiles) << 5) + int64_t(idx) * kSweepRows;
        for (int r0 = 0; r0 < kSweepRows; r0 += 32 * kI) {
            int v[kI];
#pragma unroll
            for (int k = 0; k < kI; ++k) {
                const int64_t i = base + r0 + 32 * k + lane;
                v[k] = i < n ? __ldg(J.perm + i) : -1;
            }
#pragma unroll
            for (int k = 0; k < kI; ++k) {
                if (v[k] < 0) continue;
                typename Rows<T>::Extra ex;
                Rows<T>::load_extra(ex, J.rinv, v[k]);
                Rows<T>::update(R(0), a, c, __ldg(J.outdeg + v[k]), wc[v[k]], ex, wn + v[k], f);
            }
        }
        return;
    }
    const WS *wc = wb[s.wsel];
    R *ranks = static_cast<R *>(J.ranks);
    for (int r0 = 0; r0 < kSweepRows; r0 += 32 * kI) {
        int32_t od[kI];
        WS w[kI];
#pragma unroll
        for (int k = 0; k < kI; ++k) {
            const int64_t v = int64_t(idx) * kSweepRows + r0 + 32 * k + lane;
            od[k] = v < n ? __ldg(J.outdeg + v) : 0;
            w[k] = v < n ? wc[v] : WS{};
        }
#pragma unroll
        for (int k = 0; k < kI; ++k) {
            const int64_t v = int64_t(idx) * kSweepRows + r0 + 32 * k + lane;
            if (v >= n) continue;
            if (s.mode == kSwSum) f.s += Rows<T>::fix_x(w[k], od[k]);
            else ranks[v] = static_cast<R>(Rows<T>::x_of(w[k], od[k]) * s.inv_s);
        }
    }
}

// a warp's sums of one job into the job's accumulator of this phase
__device__ __forceinline__ void sweep_flush(const JobDev *sjd, int job, int buf, Fix3 &f,
                                            int lane) {
    if (job < 0) return;
    const long long r = warp_sum_ll(f.r), d = warp_sum_ll(f.d), s = warp_sum_ll(f.s);
    if (lane == 0) {
        unsigned long long *acc = sjd[job].ctl->acc[buf];
        if (r) atomicAdd(acc + 0, static_cast<unsigned long long>(r));
        if (d) atomicAdd(acc + 1, static_cast<unsigned long long>(d));
        if (s) atomicAdd(acc + 2, static_cast<unsigned long long>(s));
    }
    f = Fix3{};
}

// the next batch of units for this warp: from its block's share while it
// lasts, then from another block's share that has units left (lanes look at
// the blocks in parallel); returns [*u0, *u1), empty when the phase's work
// is all claimed
__device__ void sweep_claim(const SweepArgs &A, int parity, int phase, int own_start,
                            int own_len, bool &own_left, int *u0, int *u1, int lane) {
    int a = 0, b = 0;
    if (own_left) {
        int k = 0;
        if (lane == 0) k = atomicAdd(A.ctr + parity * A.nb + blockIdx.x, kSweepClaim);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k < own_len) {
            *u0 = own_start + k;
            *u1 = own_start + (k + kSweepClaim < own_len ? k + kSweepClaim : own_len);
            return;
        }
        own_left = false;
    }
    for (int attempt = 0; attempt < 64; ++attempt) {
        int cand = -1, cstart = 0, clen = 0;
        for (int i = lane; i < A.nb && cand < 0; i += 32) {
            const int v = (blockIdx.x + 1 + i) % A.nb;
            const SweepRange *rg = A.ranges + parity * A.nb + v;
            if (ld_acquire(reinterpret_cast<const unsigned *>(&rg->tag)) != unsigned(phase))
                continue;
            const int len = *(volatile const int *)&rg->len;
            if (*(volatile const int *)(A.ctr + parity * A.nb + v) < len) {
                cand = v;
                cstart = *(volatile const int *)&rg->start;
                clen = len;
            }
        }
        const unsigned any = __ballot_sync(0xffffffffu, cand >= 0);
        if (!any) break;
        const int src = __ffs(any) - 1;
        const int v = __shfl_sync(0xffffffffu, cand, src);
        const int vs = __shfl_sync(0xffffffffu, cstart, src);
        const int vl = __shfl_sync(0xffffffffu, clen, src);
        int k = 0;
        if (lane == 0) k = atomicAdd(A.ctr + parity * A.nb + v, kSweepClaim);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k < vl) {
            a = vs + k;
            b = vs + (k + kSweepClaim < vl ? k + kSweepClaim : vl);
            break;
        }
    }
    *u0 = a;
    *u1 = b;
}

template <typename T, int W>
__global__ void __launch_bounds__(32 * W, 1) k_pagerank_sweep(const SweepArgs A) {
    extern __shared__ __align__(128) unsigned char s_dyn[];
    Stream st = make_stream<W>(s_dyn);
    using R = typename Rows<T>::Real;
    using WS = typename Rows<T>::W;
    JobDev *sjd = reinterpret_cast<JobDev *>(s_dyn + pr_smem_bytes<W>());
    SwJob *sj = reinterpret_cast<SwJob *>(sjd + A.n_jobs);
    int *spre = reinterpret_cast<int *>(sj + A.n_jobs);
    __shared__ int s_ok, s_start, s_len;
    __shared__ int s_wsum[W];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nj = A.n_jobs;

    // the job table and every job's first state
    for (int j = threadIdx.x; j < nj; j += blockDim.x) {
        sjd[j] = A.jobs[j];
        const JobDev &J = sjd[j];
        SwJob s;
        s.res = s.prev_res = __longlong_as_double(0x7ff0000000000000LL);
        s.inv_s = 1.0;
        s.c = 0.0;
        s.mode = kSwInit;
        s.it = s.converged = s.wsel = 0;
        const int64_t act = J.apre[J.n] - J.apre[0];
        s.ntiles = static_cast<int>((act + 31) >> 5);
        const int64_t rest = J.n - (int64_t(s.ntiles) << 5);
        s.nempty = rest > 0 ? static_cast<int>((rest + kSweepRows - 1) / kSweepRows) : 0;
        s.nrows = static_cast<int>((J.n + kSweepRows - 1) / kSweepRows);
        s.units = 0;
        sj[j] = s;
    }
    __syncthreads();

    for (int phase = 0;; ++phase) {
        const int buf = phase % 3, parity = phase & 1;
        // advance every job on the sums of the previous phase
        for (int j = threadIdx.x; j < nj; j += blockDim.x) {
            SwJob &s = sj[j];
            const JobDev &J = sjd[j];
            if (phase > 0 && s.mode != kSwDone) {
                const unsigned long long *acc = J.ctl->acc[(phase - 1) % 3];
                if (s.mode == kSwInit) {
                    s.c = teleport(J.alpha, __ldcg(acc + 1), J.n);
                    s.mode = kSwIter;
                } else if (s.mode == kSwIter) {
                    const double r = static_cast<double>(__ldcg(acc + 0)) / kFix;
                    s.prev_res = s.res;
                    s.res = r;
                    ++s.it;
                    s.wsel ^= 1;
                    bool stop = false;
                    if (r < J.tol) s.converged = 1, stop = true;
                    else if (sizeof(R) == 4 && r >= s.prev_res) s.converged = 1, stop = true;
                    else if (s.it >= J.max_iter) stop = true;
                    if (stop) s.mode = kSwSum;
                    else s.c = teleport(J.alpha, __ldcg(acc + 1), J.n);
                } else if (s.mode == kSwSum) {
                    s.inv_s = 1.0 / (static_cast<double>(__ldcg(acc + 2)) / kFix);
                    s.mode = kSwWrite;
                } else {  // the ranks are written
                    s.mode = kSwDone;
                    if (blockIdx.x == 0) {
                        J.ctl->iters = s.it;
                        J.ctl->residual = s.res;
                        J.ctl->converged = s.converged;
                        J.ctl->nblocks = A.nb;
                    }
                }
            }
            s.units = s.mode == kSwIter ? s.ntiles + s.nempty
                      : s.mode == kSwDone ? 0
                                          : s.nrows;
            // the accumulator of the next phase starts at zero; its last
            // readers passed the previous barrier
            if (blockIdx.x == 0) {
                unsigned long long *nx = J.ctl->acc[(phase + 1) % 3];
                nx[0] = nx[1] = nx[2] = 0;
            }
        }
        __syncthreads();
        // first unit of every job (exclusive scan, consecutive jobs per thread)
        {
            const int per = (nj + blockDim.x - 1) / blockDim.x;
            const int j0 = threadIdx.x * per;
            int tot = 0;
            for (int j = j0; j < j0 + per && j < nj; ++j) tot += sj[j].units;
            int incl = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            if (lane == 31) s_wsum[warp] = incl;
            __syncthreads();
            int before = 0;
            for (int w = 0; w < warp; ++w) before += s_wsum[w];
            int run = before + incl - tot;
            for (int j = j0; j < j0 + per && j < nj; ++j) {
                spre[j] = run;
                run += sj[j].units;
            }
            if (threadIdx.x == blockDim.x - 1) spre[nj] = before + incl;
        }
        __syncthreads();
        const int total = spre[nj];
        if (total == 0) break;  // every job is done
        if (threadIdx.x == 0) {
            const int a = static_cast<int>(int64_t(total) * blockIdx.x / A.nb);
            const int b = static_cast<int>(int64_t(total) * (blockIdx.x + 1) / A.nb);
            s_start = a;
            s_len = b - a;
            SweepRange *rg = A.ranges + parity * A.nb + blockIdx.x;
            rg->start = a;
            rg->len = b - a;
            __threadfence();
            atomicExch(&rg->tag, phase);
            A.ctr[(parity ^ 1) * A.nb + blockIdx.x] = 0;  // the next phase's counter
        }
        __syncthreads();

        // the units: a pipeline of tiles (the next tile's head and row data
        // and its first descriptor segment load while the current one is
        // summed); chunks are done as they come
        bool own_left = true;
        int q0 = 0, q1 = 0;   // this warp's claimed, not yet taken units
        int acc_job = -1;
        Fix3 facc;
        bool failed = false;
        const int own_start = s_start, own_len = s_len;
        auto next = [&](int hint) -> SwUnit {
            if (q0 == q1) sweep_claim(A, parity, phase, own_start, own_len, own_left, &q0, &q1,
                                      lane);
            const int u = q0 < q1 ? q0++ : -1;
            return sweep_unit(u, spre, sj, nj, hint);
        };
        SwUnit u0 = next(0);
        SwUnit u1 = next(u0.job);
        TileInfo<T> cur, nxt;
        bool cur_row = false;
        if (u0.kind == 1) cur = load_head<T>(u0.idx, static_cast<int>(sjd[u0.job].n),
                                             sjd[u0.job].tinfo, sjd[u0.job].perm, lane);
        if (u1.kind == 1) nxt = load_head<T>(u1.idx, static_cast<int>(sjd[u1.job].n),
                                             sjd[u1.job].tinfo, sjd[u1.job].perm, lane);
        while (u0.kind != 0 && !failed) {
            const JobDev &J0 = sjd[u0.job];
            const SwJob &s0 = sj[u0.job];
            if (u0.job != acc_job) {
                sweep_flush(sjd, acc_job, buf, facc, lane);
                acc_job = u0.job;
            }
            WS *wb0[2] = {static_cast<WS *>(J0.w0), static_cast<WS *>(J0.w1)};
            if (u0.kind == 2) {
                sweep_chunk<T>(J0, s0, u0.idx - (s0.mode == kSwIter ? s0.ntiles : 0), facc,
                               lane);
                u0 = u1;
                cur = nxt;
                cur_row = false;
                u1 = next(u0.job);
                if (u1.kind == 1) nxt = load_head<T>(u1.idx, static_cast<int>(sjd[u1.job].n),
                                                     sjd[u1.job].tinfo, sjd[u1.job].perm, lane);
                continue;
            }
            if (!cur_row) load_row<T>(cur, J0.outdeg, wb0[s0.wsel], J0.rinv);
            const SwUnit u2 = next(u1.kind ? u1.job : u0.job);
            if (u1.kind == 1) {
                const JobDev &J1 = sjd[u1.job];
                WS *w1c = static_cast<WS *>(sj[u1.job].wsel ? J1.w1 : J1.w0);
                load_row<T>(nxt, J1.outdeg, w1c, J1.rinv);
            }
            TileInfo<T> nx2;
            if (u2.kind == 1) nx2 = load_head<T>(u2.idx, static_cast<int>(sjd[u2.job].n),
                                                 sjd[u2.job].tinfo, sjd[u2.job].perm, lane);
            const int v = cur.v;
            const WS *wc = wb0[s0.wsel];
            R sum = R(0);
            const bool next_tile = u1.kind == 1 && nxt.cnt > 0;
            const uint2 *dn = next_tile ? sjd[u1.job].desc + size_t(nxt.d8) * kU : nullptr;
            if (!tile_sum<T>(J0.desc + size_t(cur.d8) * kU, cur.cnt, dn, next_tile ? nxt.cnt : 0,
                             next_tile, st, wc + (v < 0 ? 0 : v), 1u << lane,
                             gather_bounds(v, J0.n), lane, sum)) {
                failed = true;
                break;
            }
            if (v >= 0)
                Rows<T>::update(sum, static_cast<R>(J0.alpha), static_cast<R>(s0.c), cur.od,
                                cur.wv, cur.ex, wb0[s0.wsel ^ 1] + v, facc);
            u0 = u1;
            cur = nxt;
            cur_row = u0.kind == 1;
            u1 = u2;
            nxt = nx2;
        }
        if (failed) {
            st.drain();
            if (lane == 0) atomicCAS(&A.ctl->status, 0, (int)FFG_ERR_TIMEOUT);
        } else if (st.issued) {
            st.drain();
        }
        st.issued = false;
        sweep_flush(sjd, acc_job, buf, facc, lane);
        if (!sweep_barrier(A.ctl, unsigned(phase + 1) * unsigned(A.nb), &s_ok)) break;
    }
    // a failure: every unfinished job reports it
    if (blockIdx.x == 0 && *(volatile int *)&A.ctl->status != 0)
        for (int j = threadIdx.x; j < nj; j += blockDim.x)
            if (sj[j].mode != kSwDone) atomicCAS(&sjd[j].ctl->status, 0, A.ctl->status);
}

// Layout kernels over every distinct graph of a batch: a global row or tile
// index -> graph by binary search over the graphs' first rows or tiles.
struct GraphDev {
    const int64_t *in_ptr;
    const int32_t *in_idx;
    uint2 *desc;
    int32_t *cnt;
    uint2 *tinfo;
    int32_t *perm;
    int32_t *aflag;  // this graph's part of the batch's row flags
    int64_t *apre;   // ... and of their prefix sums
    int64_t n, e;
    int64_t tile0;   // first global tile of this graph
    int64_t row0;    // first global row of this graph
};

__device__ __forceinline__ int graph_of(const GraphDev *__restrict__ gr, int n_graphs, int64_t x,
                                        bool by_tile) {
    int lo = 0, hi = n_graphs - 1;  // last graph starting at or before x
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((by_tile ? gr[mid].tile0 : gr[mid].row0) <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void k_active_flags_batch(const GraphDev *__restrict__ gr, int n_graphs,
                                     int64_t total_rows) {
    for (int64_t x = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; x < total_rows;
         x += int64_t(gridDim.x) * blockDim.x) {
        const GraphDev &g = gr[graph_of(gr, n_graphs, x, false)];
        active_flag(g.in_ptr, x - g.row0, g.aflag);
    }
}
__global__ void k_perm_batch(const GraphDev *__restrict__ gr, int n_graphs, int64_t total_rows) {
    for (int64_t x = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; x < total_rows;
         x += int64_t(gridDim.x) * blockDim.x) {
        const GraphDev &g = gr[graph_of(gr, n_graphs, x, false)];
        place_row(g.apre, g.n, x - g.row0, g.perm);
    }
}
__global__ void __launch_bounds__(kLayoutThreads) k_pr_layout_batch(const GraphDev *__restrict__ gr,
                                                                     int n_graphs,
                                                                     int64_t total_tiles) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t step = int64_t(gridDim.x) * (kLayoutThreads / 32);
    for (int64_t gt = int64_t(blockIdx.x) * (kLayoutThreads / 32) + warp; gt < total_tiles;
         gt += step) {
        const GraphDev g = gr[graph_of(gr, n_graphs, gt, true)];
        layout_tile(g.in_ptr, g.in_idx, g.perm, g.n, g.e, 0, 0, g.desc, g.cnt, g.tinfo,
                    gt - g.tile0, lane);
    }
}

unsigned grid_for(int64_t items, int per_block, int sms) {
    const int64_t want = (items + per_block - 1) / per_block;
    const int64_t cap = int64_t(sms) * 32;
    return static_cast<unsigned>(want < 1 ? 1 : (want < cap ? want : cap));
}

ffg_status device_sms(int *sms) {
    int dev = 0;
    FFG_TRY(check_cuda(cudaGetDevice(&dev), "cudaGetDevice"));
    return check_cuda(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev), "attr");
}

// slots (rows with in-edges first), descriptors, tile cost prefix
ffg_status launch_layout(const ffg_graph *g, PrWs &w, cudaStream_t stream) {
    int sms = 0;
    FFG_TRY(device_sms(&sms));
    const int64_t n = g->n_nodes;
    const int64_t tiles = (n + 31) / 32;
    k_active_flags<<<grid_for(n, 256, sms), 256, 0, stream>>>(g->in_ptr, n, w.aflag);
    count_launch();
    FFG_TRY(check_launch("k_active_flags"));
    FFG_TRY(scan_exclusive(w.aflag, w.apre, n, w.ascan, stream));
    k_perm<<<grid_for(n, 256, sms), 256, 0, stream>>>(w.apre, n, w.perm);
    count_launch();
    FFG_TRY(check_launch("k_perm"));
    k_pr_layout<<<grid_for(tiles, kLayoutThreads / 32, sms), kLayoutThreads, 0, stream>>>(
        g->in_ptr, g->in_idx, w.perm, n, g->n_edges, 0, 0, w.desc, w.cnt, w.tinfo);
    count_launch();
    FFG_TRY(check_launch("k_pr_layout"));
    return scan_exclusive(w.cnt, w.tpre, tiles, w.scan, stream);
}

// co-resident blocks per SM of kernel `kern` (W warps per block); sets its
// dynamic shared memory limit
template <int W>
ffg_status kernel_config(const void *kern, int *blocks_per_sm, int *sms) {
    int dev = 0;
    FFG_TRY(check_cuda(cudaGetDevice(&dev), "cudaGetDevice"));
    FFG_TRY(check_cuda(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev), "attr"));
    const size_t smem = pr_smem_bytes<W>();
    FFG_TRY(check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            static_cast<int>(smem)),
                       "smem attribute"));
    FFG_TRY(check_cuda(
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, 32 * W, smem),
        "occupancy"));
    if (*blocks_per_sm < 1) return set_error("kernel does not fit on the device"), FFG_ERR_CUDA;
    return FFG_OK;
}

template <typename T, int W>
ffg_status launch_single(const JobDev &single, int nb, cudaStream_t stream) {
    const size_t smem = pr_smem_bytes<W>();
    JobDev s = single;
    void *args[] = {(void *)&s};
    FFG_TRY(check_cuda(cudaLaunchCooperativeKernel((const void *)k_pagerank<T, W>, dim3(nb),
                                                   dim3(32 * W), args, smem, stream),
                       "k_pagerank"));
    count_launch();
    return FFG_OK;
}

template <typename T, int W>
ffg_status launch_pr(const JobDev *jobs, const int2 *items, const int *first, int *queue,
                     int n_items, int nb, cudaStream_t stream) {
    const size_t smem = pr_smem_bytes<W>();
    void *args[] = {(void *)&jobs, (void *)&items, (void *)&first, (void *)&queue,
                    (void *)&n_items};
    FFG_TRY(check_cuda(cudaLaunchCooperativeKernel((const void *)k_pagerank_batch<T, W>,
                                                   dim3(nb), dim3(32 * W), args, smem, stream),
                       "k_pagerank_batch"));
    count_launch();
    return FFG_OK;
}

template <typename T, int W>
ffg_status launch_pr_param(const BatchParams &P, int nb, cudaStream_t stream) {
    const size_t smem = pr_smem_bytes<W>();
    void *args[] = {(void *)&P};
    FFG_TRY(check_cuda(cudaLaunchCooperativeKernel((const void *)k_pagerank_batch_p<T, W>,
                                                   dim3(nb), dim3(32 * W), args, smem, stream),
                       "k_pagerank_batch_p"));
    count_launch();
    return FFG_OK;
}

template <typename T>
ffg_status launch(const ffg_graph *g, double alpha, double tol, int max_iter, int init,
                  void *ranks, PrWs &w, cudaStream_t stream) {
    // the FP64 forms hide their longer (16-byte or converted) gathers with
    // more warps; FP32 is faster with more registers per warp
    constexpr int W = sizeof(typename Rows<T>::Real) == 8 ? kWarpsSingle64 : kWarpsSingle;
    int per_sm = 0, sms = 0;
    FFG_TRY((kernel_config<W>((const void *)k_pagerank<T, W>, &per_sm, &sms)));
    const int64_t tiles = (g->n_nodes + 31) / 32;
    int64_t max_res = int64_t(sms) * per_sm;
    if (max_res > kMaxBlocks) max_res = kMaxBlocks;
    const int64_t want = (tiles + 4 * W - 1) / (4 * W);  // >= ~4 tiles per warp
    const int nb = static_cast<int>(want < 1 ? 1 : (want > max_res ? max_res : want));
    JobDev J;
    J.outdeg = g->outdeg;
    J.desc = w.desc;
    J.tinfo = w.tinfo;
    J.perm = w.perm;
    J.tpre = w.tpre;
    J.apre = w.apre;
    J.ranks = ranks;
    J.w0 = w.w0;
    J.w1 = w.w1;
    J.rinv = w.rinv;
    J.ctl = w.ctl;
    J.n = g->n_nodes;
    J.alpha = alpha;
    J.tol = tol;
    J.max_iter = max_iter;
    J.init = init;
    J.group = nb;
    J.pad = 0;
    return launch_single<T, W>(J, nb, stream);
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
    return carve(nullptr, n_nodes, n_edges, prec).bytes;
}

extern "C" ffg_status pagerank_solve(const ffg_graph *g, double damping, double tol,
                                     int32_t max_iter, ffg_prec prec, void *ranks, int init,
                                     void *workspace, size_t ws_bytes, int32_t *iters_out,
                                     double *residual_out, void *stream_) {
    clear_error();
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (!g || g->n_nodes <= 0 || !g->in_ptr || !g->outdeg || (g->n_edges > 0 && !g->in_idx))
        return set_error("graph is empty or incomplete"), FFG_ERR_INVALID_ARG;
    if (g->n_nodes >= (int64_t(1) << 31) || !desc_fits(g->n_nodes, g->n_edges))
        return set_error("too many nodes or edges"), FFG_ERR_OVERFLOW;
    if (!(damping > 0.0 && damping < 1.0))
        return set_error("damping must lie in (0,1)"), FFG_ERR_INVALID_ARG;
    if (!(tol >= 0.0) || max_iter < 1 || max_iter > FFG_MAX_ITER)
        return set_error("tol must be >= 0 and max_iter in [1, %d]", FFG_MAX_ITER),
               FFG_ERR_INVALID_ARG;
    if (prec != FFG_F64 && prec != FFG_F32)
        return set_error("unknown precision %d", (int)prec), FFG_ERR_INVALID_ARG;
    if (!ranks || !workspace) return set_error("ranks/workspace NULL"), FFG_ERR_INVALID_ARG;
    if (!aligned256(workspace))
        return set_error("workspace not 256-byte aligned"), FFG_ERR_INVALID_ARG;
    PrWs w = carve(workspace, g->n_nodes, g->n_edges, prec);
    if (ws_bytes < w.bytes)
        return set_error("workspace %zu bytes, need %zu", ws_bytes, w.bytes), FFG_ERR_NO_MEMORY;
    if (init & ~(FFG_INIT_RANKS | FFG_INIT_LAYOUT))
        return set_error("unknown init flags 0x%x", init), FFG_ERR_INVALID_ARG;
    FFG_TRY(check_cuda(cudaMemsetAsync(w.ctl, 0, sizeof(PrCtl), stream), "memset"));
    if (!(init & FFG_INIT_LAYOUT)) FFG_TRY(launch_layout(g, w, stream));
    const int warm = (init & FFG_INIT_RANKS) ? 1 : 0;
    if (prec == FFG_F32)
        FFG_TRY(launch<float>(g, damping, tol, max_iter, warm, ranks, w, stream));
    else if (g->n_nodes <= kFxMaxNodes)
        FFG_TRY(launch<F64x>(g, damping, tol, max_iter, warm, ranks, w, stream));
    else
        FFG_TRY(launch<double>(g, damping, tol, max_iter, warm, ranks, w, stream));
    if (!iters_out && !residual_out) return FFG_OK;
    return read_result(w.ctl, iters_out, residual_out, stream);
}

extern "C" ffg_status pagerank_prepare(const ffg_graph *g, ffg_prec prec, void *workspace,
                                       size_t ws_bytes, void *stream_) {
    clear_error();
    if (!g || g->n_nodes <= 0 || !g->in_ptr || (g->n_edges > 0 && !g->in_idx))
        return set_error("graph is empty or incomplete"), FFG_ERR_INVALID_ARG;
    if (g->n_nodes >= (int64_t(1) << 31) || !desc_fits(g->n_nodes, g->n_edges))
        return set_error("too many nodes or edges"), FFG_ERR_OVERFLOW;
    if (prec != FFG_F64 && prec != FFG_F32)
        return set_error("unknown precision %d", (int)prec), FFG_ERR_INVALID_ARG;
    if (!workspace || !aligned256(workspace))
        return set_error("workspace NULL or not 256-byte aligned"), FFG_ERR_INVALID_ARG;
    PrWs w = carve(workspace, g->n_nodes, g->n_edges, prec);
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
// PageRank over a range of rows: the row-partitioned form of the solve.  A
// rank owns rows [row0, row1); per iteration it forms w' of its rows from w
// of every row, and the ranks exchange their rows of w' and their
// fixed-point sums between iterations (host side).  One launch per
// iteration, no grid barrier: the exchange is the synchronisation.
// ---------------------------------------------------------------------------
namespace ffg {
namespace {

struct RowsWs {
    double *rinv;   // FP64: 1 / outdeg per row of the range
    uint2 *desc;
    int32_t *cnt;
    uint2 *tinfo;
    int64_t *tpre;
    int64_t *scan;
    int32_t *perm;
    int32_t *aflag;
    int64_t *apre;
    int64_t *ascan;
    size_t bytes;
};

// The descriptors come last, so that every table's place depends on the
// number of rows only: an iteration finds them without knowing the range's
// in-edges (which would take a device read).
RowsWs carve_rows(void *base, int64_t n, int64_t e) {
    Carver c(base);
    RowsWs w;
    const int64_t tiles = (n + 31) / 32;
    w.rinv = c.take<double>(size_t(n));
    w.cnt = c.take<int32_t>(size_t(tiles));
    w.tinfo = c.take<uint2>(size_t(tiles));
    w.tpre = c.take<int64_t>(size_t(tiles) + 1);
    w.scan = c.take<int64_t>(size_t(scan_scratch_elems(tiles)));
    w.perm = c.take<int32_t>(size_t(n));
    w.aflag = c.take<int32_t>(size_t(n));
    w.apre = c.take<int64_t>(size_t(n) + 1);
    w.ascan = c.take<int64_t>(size_t(scan_scratch_elems(n)));
    w.desc = c.take<uint2>(size_t(desc_capacity(n, e)));
    w.bytes = c.off;
    return w;
}

// One range's view: rows are local (0 .. n-1, global row0 + local), w
// pointers are shifted by row0 so that local rows index them directly.
struct RowsDev {
    const int32_t *outdeg;  // of the range's rows
    const uint2 *desc;
    const uint2 *tinfo;
    const int32_t *perm;
    const int64_t *apre;
    double *rinv;
    const void *w_in;       // w of every row, shifted by row0
    void *w_out;            // w' of every row, shifted by row0
    void *ranks;            // shifted by row0
    unsigned long long *sums;
    ffg_rows_ctl *ctl;      // the solve's state: dangling mass, scale, decisions
    int64_t n, n_all;       // rows of the range, of the graph
    int64_t row0;           // the range's first row
    double alpha;
};

template <int W>
__device__ __forceinline__ void add_sums(const RowsDev &R, const Fix3 &f) {
    const Fix3 b = block_sum_fix<W>(f);
    if (threadIdx.x == 0) {
        if (b.r) atomicAdd(R.sums + 0, static_cast<unsigned long long>(b.r));
        if (b.d) atomicAdd(R.sums + 1, static_cast<unsigned long long>(b.d));
        if (b.s) atomicAdd(R.sums + 2, static_cast<unsigned long long>(b.s));
    }
}

// w of the range's rows from the start vector (ranks, or 1/n_all), the
// per-row reciprocals, and the range's dangling mass
template <typename T>
__global__ void __launch_bounds__(256) k_rows_init(const RowsDev R) {
    using WS = typename Rows<T>::W;
    using Rr = typename Rows<T>::Real;
    WS *wo = static_cast<WS *>(R.w_out);
    const Rr *x = static_cast<const Rr *>(R.ranks);
    const double inv_n = 1.0 / static_cast<double>(R.n_all);
    Fix3 f;
    for (int64_t v = int64_t(blockIdx.x) * 256 + threadIdx.x; v < R.n;
         v += int64_t(gridDim.x) * 256) {
        const double x0 = x ? static_cast<double>(x[v]) : inv_n;
        const int32_t od = __ldg(R.outdeg + v);
        wo[v] = Rows<T>::init(x0, od);
        Rows<T>::store_rinv(R.rinv, v, od);
        if (od == 0) f.d += to_fix(x0);
    }
    add_sums<8>(R, f);
}

// one iteration over the range's tiles (each warp takes every nw-th tile,
// the next one loaded while the current one is summed), then its rows
// without in-edges; sums[3] counts bounded waits that expired
template <typename T, int W>
__global__ void __launch_bounds__(32 * W, 1) k_rows_step(const RowsDev R) {
    extern __shared__ __align__(128) unsigned char s_dyn[];
    Stream st = make_stream<W>(s_dyn);
    using WS = typename Rows<T>::W;
    using Rr = typename Rows<T>::Real;
    const WS *wc = static_cast<const WS *>(R.w_in);
    WS *wn = static_cast<WS *>(R.w_out);
    const int lane = threadIdx.x & 31;
    const int64_t gw = int64_t(blockIdx.x) * W + (threadIdx.x >> 5);
    const int64_t nw = int64_t(gridDim.x) * W;
    const int ni = static_cast<int>(R.n);
    const int64_t ntiles = (R.apre[R.n] - R.apre[0] + 31) >> 5;
    const Rr a = static_cast<Rr>(R.alpha);
    const Rr c = static_cast<Rr>(teleport(R.alpha, R.ctl->dangling, R.n_all));
    Fix3 f;
    bool failed = false;
    if (gw < ntiles) {
        int t = static_cast<int>(gw);
        TileInfo<T> cur = load_head<T>(t, ni, R.tinfo, R.perm, lane);
        load_row<T>(cur, R.outdeg, wc, R.rinv);
        while (true) {
            const int64_t tn = t + nw;
            const bool has_next = tn < ntiles;
            TileInfo<T> nxt = load_head<T>(has_next ? static_cast<int>(tn) : t, ni, R.tinfo,
                                           R.perm, lane);
            if (has_next) load_row<T>(nxt, R.outdeg, wc, R.rinv);
            const int v = cur.v;
            Rr sum = Rr(0);
            if (!tile_sum<T>(R.desc, cur, nxt, has_next, st, wc + (v < 0 ? 0 : v), 1u << lane,
                             gather_bounds(v < 0 ? v : R.row0 + v, R.n_all), lane, sum)) {
                failed = true;
                break;
            }
            if (v >= 0) Rows<T>::update(sum, a, c, cur.od, cur.wv, cur.ex, wn + v, f);
            if (!has_next) break;
            cur = nxt;
            t = static_cast<int>(tn);
        }
    }
    if (failed || st.issued) st.drain();
    // rows without in-edges: x' = c
    const int64_t slot_empty = ntiles << 5;
    for (int64_t i = slot_empty + int64_t(blockIdx.x) * 32 * W + threadIdx.x; i < R.n;
         i += int64_t(gridDim.x) * 32 * W) {
        const int v = __ldg(R.perm + i);
        typename Rows<T>::Extra ex;
        Rows<T>::load_extra(ex, R.rinv, v);
        Rows<T>::update(Rr(0), a, c, __ldg(R.outdeg + v), wc[v], ex, wn + v, f);
    }
    add_sums<W>(R, f);
    if (failed && lane == 0) atomicAdd(R.sums + 3, 1ULL);
}

// sum of x over the range (sums[2]), or, with ranks set, x * scale into ranks
template <typename T>
__global__ void __launch_bounds__(256) k_rows_finish(const RowsDev R) {
    using WS = typename Rows<T>::W;
    using Rr = typename Rows<T>::Real;
    const WS *wc = static_cast<const WS *>(R.w_in);
    Rr *x = static_cast<Rr *>(R.ranks);
    Fix3 f;
    for (int64_t v = int64_t(blockIdx.x) * 256 + threadIdx.x; v < R.n;
         v += int64_t(gridDim.x) * 256) {
        const int32_t od = __ldg(R.outdeg + v);
        if (x) x[v] = static_cast<Rr>(Rows<T>::x_of(wc[v], od) * R.ctl->scale);
        else f.s += Rows<T>::fix_x(wc[v], od);
    }
    if (!x) add_sums<8>(R, f);
}

// The solve's control between operations (one thread): the stopping rule
// and the normalisation of pagerank_solve (advance() and the epilogue of
// run_job), taken from the fixed-point sums of every rank; the sums used are
// cleared for the next operation.
__global__ void k_rows_ctl(ffg_rows_ctl *ctl, unsigned long long *sums, int op, double tol,
                           int max_iter, int fp32) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (op == FFG_ROWS_INIT) {
        ctl->iters = ctl->stop = ctl->converged = ctl->status = 0;
        ctl->residual = ctl->prev_residual = __longlong_as_double(0x7ff0000000000000LL);
        ctl->scale = 1.0;
        ctl->dangling = 0;
        return;
    }
    if (op == FFG_ROWS_START) {
        ctl->dangling = sums[1];
    } else if (op == FFG_ROWS_ADVANCE) {
        const double r = static_cast<double>(sums[0]) / kFix;
        ctl->prev_residual = ctl->residual;
        ctl->residual = r;
        ctl->dangling = sums[1];
        ++ctl->iters;
        if (sums[3]) {
            ctl->status = FFG_ERR_TIMEOUT;
            ctl->stop = 1;
        } else if (r < tol) {
            ctl->converged = ctl->stop = 1;
        } else if (fp32 && r >= ctl->prev_residual) {
            ctl->converged = ctl->stop = 1;
        } else if (ctl->iters >= max_iter) {
            ctl->stop = 1;
        }
    } else {  // FFG_ROWS_SCALE
        ctl->scale = 1.0 / (static_cast<double>(sums[2]) / kFix);
    }
    sums[0] = sums[1] = sums[2] = sums[3] = 0;
}

ffg_status rows_check(const ffg_graph *g, int64_t row0, int64_t row1, ffg_prec prec) {
    if (!g || g->n_nodes <= 0 || !g->in_ptr || !g->outdeg || (g->n_edges > 0 && !g->in_idx))
        return set_error("graph is empty or incomplete"), FFG_ERR_INVALID_ARG;
    if (g->n_nodes >= (int64_t(1) << 31)) return set_error("too many nodes"), FFG_ERR_OVERFLOW;
    if (!(0 <= row0 && row0 < row1 && row1 <= g->n_nodes))
        return set_error("rows [%lld, %lld) outside [0, %lld)", (long long)row0,
                         (long long)row1, (long long)g->n_nodes),
               FFG_ERR_INVALID_ARG;
    if (prec != FFG_F64 && prec != FFG_F32)
        return set_error("unknown precision %d", (int)prec), FFG_ERR_INVALID_ARG;
    return FFG_OK;
}

// in-edges of the range: in_ptr[row0] and in_ptr[row1] (a synchronous read)
ffg_status rows_edges(const ffg_graph *g, int64_t row0, int64_t row1, int64_t *ebase,
                      int64_t *eend) {
    FFG_TRY(check_cuda(cudaMemcpy(ebase, g->in_ptr + row0, sizeof(int64_t),
                                  cudaMemcpyDeviceToHost), "read in_ptr"));
    FFG_TRY(check_cuda(cudaMemcpy(eend, g->in_ptr + row1, sizeof(int64_t),
                                  cudaMemcpyDeviceToHost), "read in_ptr"));
    if (!(0 <= *ebase && *ebase <= *eend && *eend <= g->n_edges))
        return set_error("in_ptr is not a row-pointer array"), FFG_ERR_INVALID_ARG;
    if (!desc_fits(row1 - row0, *eend - *ebase))
        return set_error("too many edges in the range"), FFG_ERR_OVERFLOW;
    return FFG_OK;
}

}  // namespace
}  // namespace ffg

extern "C" size_t pagerank_rows_w_bytes(ffg_prec prec) {
    return prec == FFG_F32 ? sizeof(float) : prec == FFG_F64 ? sizeof(Fx) : 0;
}

extern "C" size_t pagerank_rows_workspace_bytes(const ffg_graph *g, int64_t row0, int64_t row1,
                                                ffg_prec prec) {
    clear_error();
    int64_t eb = 0, ee = 0;
    if (rows_check(g, row0, row1, prec) != FFG_OK || rows_edges(g, row0, row1, &eb, &ee) != FFG_OK)
        return 0;
    return carve_rows(nullptr, row1 - row0, ee - eb).bytes;
}

extern "C" ffg_status pagerank_rows_prepare(const ffg_graph *g, int64_t row0, int64_t row1,
                                            ffg_prec prec, void *workspace, size_t ws_bytes,
                                            void *stream_) {
    clear_error();
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    FFG_TRY(rows_check(g, row0, row1, prec));
    if (!workspace || !aligned256(workspace))
        return set_error("workspace NULL or not 256-byte aligned"), FFG_ERR_INVALID_ARG;
    int64_t eb = 0, ee = 0;
    FFG_TRY(rows_edges(g, row0, row1, &eb, &ee));
    const int64_t n = row1 - row0, tiles = (n + 31) / 32;
    RowsWs w = carve_rows(workspace, n, ee - eb);
    if (ws_bytes < w.bytes)
        return set_error("workspace %zu bytes, need %zu", ws_bytes, w.bytes), FFG_ERR_NO_MEMORY;
    int sms = 0;
    FFG_TRY(device_sms(&sms));
    const int64_t *in_ptr = g->in_ptr + row0;
    k_active_flags<<<grid_for(n, 256, sms), 256, 0, stream>>>(in_ptr, n, w.aflag);
    count_launch();
    FFG_TRY(check_launch("k_active_flags"));
    FFG_TRY(scan_exclusive(w.aflag, w.apre, n, w.ascan, stream));
    k_perm<<<grid_for(n, 256, sms), 256, 0, stream>>>(w.apre, n, w.perm);
    count_launch();
    FFG_TRY(check_launch("k_perm"));
    k_pr_layout<<<grid_for(tiles, kLayoutThreads / 32, sms), kLayoutThreads, 0, stream>>>(
        in_ptr, g->in_idx, w.perm, n, ee, eb, row0, w.desc, w.cnt, w.tinfo);
    count_launch();
    FFG_TRY(check_launch("k_pr_layout"));
    return scan_exclusive(w.cnt, w.tpre, tiles, w.scan, stream);
}

namespace ffg {
namespace {

template <typename T, int W>
ffg_status launch_rows_step(const RowsDev &R, cudaStream_t stream) {
    int per_sm = 0, sms = 0;
    FFG_TRY((kernel_config<W>((const void *)k_rows_step<T, W>, &per_sm, &sms)));
    const int64_t tiles = (R.n + 31) / 32;
    const int64_t want = (tiles + W - 1) / W;  // a tile per warp at least
    const int64_t most = int64_t(sms) * per_sm;
    const unsigned grid = static_cast<unsigned>(want < 1 ? 1 : (want < most ? want : most));
    k_rows_step<T, W><<<grid, 32 * W, pr_smem_bytes<W>(), stream>>>(R);
    count_launch();
    return check_launch("k_rows_step");
}

template <typename T>
ffg_status launch_rows(int op, const RowsDev &R, cudaStream_t stream) {
    int sms = 0;
    FFG_TRY(device_sms(&sms));
    const unsigned grid = grid_for(R.n, 256, sms);
    switch (op) {
    case FFG_ROWS_INIT:
        k_rows_init<T><<<grid, 256, 0, stream>>>(R);
        count_launch();
        return check_launch("k_rows_init");
    case FFG_ROWS_STEP:
        return launch_rows_step<T, sizeof(typename Rows<T>::Real) == 8 ? kWarpsSingle64
                                                                       : kWarpsSingle>(R, stream);
    default:
        k_rows_finish<T><<<grid, 256, 0, stream>>>(R);
        count_launch();
        return check_launch("k_rows_finish");
    }
}

}  // namespace
}  // namespace ffg

extern "C" ffg_status pagerank_rows_run(const ffg_graph *g, int64_t row0, int64_t row1,
                                        ffg_prec prec, const ffg_rows_op *op, void *workspace,
                                        size_t ws_bytes, void *stream_) {
    clear_error();
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    FFG_TRY(rows_check(g, row0, row1, prec));
    if (!op || op->op < FFG_ROWS_INIT || op->op > FFG_ROWS_SCALE || !op->sums || !op->ctl)
        return set_error("op: unknown operation, or sums or ctl NULL"), FFG_ERR_INVALID_ARG;
    if (!workspace || !aligned256(workspace))
        return set_error("workspace NULL or not 256-byte aligned"), FFG_ERR_INVALID_ARG;
    const int k = op->op;
    if ((k == FFG_ROWS_STEP || k == FFG_ROWS_SUM || k == FFG_ROWS_WRITE) && !op->w_in)
        return set_error("op %d: w_in missing", k), FFG_ERR_INVALID_ARG;
    if ((k == FFG_ROWS_INIT || k == FFG_ROWS_STEP) && !op->w_out)
        return set_error("op %d: w_out missing", k), FFG_ERR_INVALID_ARG;
    if (k == FFG_ROWS_WRITE && !op->ranks)
        return set_error("op %d: ranks missing", k), FFG_ERR_INVALID_ARG;
    if (k == FFG_ROWS_STEP && !(op->damping > 0.0 && op->damping < 1.0))
        return set_error("damping must lie in (0, 1)"), FFG_ERR_INVALID_ARG;
    if (k == FFG_ROWS_ADVANCE && (!(op->tol >= 0.0) || op->max_iter < 1))
        return set_error("tol must be >= 0 and max_iter >= 1"), FFG_ERR_INVALID_ARG;
    // the tables' places depend on the rows only (the descriptors come
    // last), so an iteration needs no device read; the full size was checked
    // by pagerank_rows_prepare
    const int64_t n = row1 - row0;
    if (ws_bytes < carve_rows(nullptr, n, 0).bytes)
        return set_error("workspace smaller than any range of %lld rows", (long long)n),
               FFG_ERR_NO_MEMORY;
    unsigned long long *sums = reinterpret_cast<unsigned long long *>(op->sums);
    if (k == FFG_ROWS_START || k == FFG_ROWS_ADVANCE || k == FFG_ROWS_SCALE) {
        k_rows_ctl<<<1, 32, 0, stream>>>(op->ctl, sums, k, op->tol, op->max_iter,
                                         prec == FFG_F32 ? 1 : 0);
        count_launch();
        return check_launch("k_rows_ctl");
    }
    if (k == FFG_ROWS_INIT) {
        k_rows_ctl<<<1, 32, 0, stream>>>(op->ctl, sums, k, 0.0, 1, 0);
        count_launch();
        FFG_TRY(check_launch("k_rows_ctl"));
    }
    const RowsWs w = carve_rows(workspace, n, 0);
    const size_t wb = pagerank_rows_w_bytes(prec);
    RowsDev R;
    R.outdeg = g->outdeg + row0;
    R.rinv = w.rinv;
    R.n = n;
    R.n_all = g->n_nodes;
    R.row0 = row0;
    R.alpha = op->damping;
    R.ctl = op->ctl;
    R.sums = sums;
    R.w_in = op->w_in ? static_cast<const char *>(op->w_in) + size_t(row0) * wb : nullptr;
    R.w_out = op->w_out ? static_cast<char *>(op->w_out) + size_t(row0) * wb : nullptr;
    const size_t rb = prec == FFG_F32 ? sizeof(float) : sizeof(double);
    R.ranks = op->ranks ? static_cast<char *>(op->ranks) + size_t(row0) * rb : nullptr;
    if (k == FFG_ROWS_SUM) R.ranks = nullptr;
    R.desc = w.desc;
    R.tinfo = w.tinfo;
    R.perm = w.perm;
    R.apre = w.apre;
    if (prec == FFG_F32) return launch_rows<float>(k, R, stream);
    return launch_rows<F64x>(k, R, stream);
}

// ---------------------------------------------------------------------------
// batched PageRank: many jobs (graph, damping, tolerance) in one persistent
// launch.  The plan assigns each job a group of blocks: jobs costing more
// than two blocks' share of the total get dedicated blocks (their first
// item on every one of them), the others run on one block each, placed by
// longest-processing-time-first on the least loaded block.
// ---------------------------------------------------------------------------
#include <string.h>

#include <algorithm>
#include <cmath>
#include <memory>
#include <numeric>
#include <queue>
#include <unordered_map>
#include <vector>

namespace ffg {
namespace {

struct PlanHost {
    int nb = 0;
    std::vector<int> group;           // per job
    int warps = kWarpsSingle;         // warps per block
    int claim = 0;                    // claim order (else per-block lists)
    std::vector<int> first;           // per-block lists: nb + 1
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
    if (g->n_nodes >= (int64_t(1) << 31) || !desc_fits(g->n_nodes, g->n_edges))
        return set_error("job %d: too many nodes or edges", idx), FFG_ERR_OVERFLOW;
    if (!(j.damping > 0.0 && j.damping < 1.0) || !(j.tol >= 0.0) || j.max_iter < 1 ||
        j.max_iter > FFG_MAX_ITER || (j.init & ~FFG_INIT_RANKS))
        return set_error("job %d: bad damping, tol, max_iter or init", idx), FFG_ERR_INVALID_ARG;
    return FFG_OK;
}

// Group sizes and the order of the items (see k_pagerank).
ffg_status make_plan(const ffg_pr_job *jobs, int n_jobs, int nb_max, int warps,
                     const ffg_pr_tuning &tu, PlanHost &P) {
    P.claim = tu.claim;
    // distinct graphs (jobs may share one)
    std::unordered_map<const int64_t *, int> gidx;
    P.graph_of_job.resize(n_jobs);
    P.warps = warps;
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
        cost[j] = tu.job_cost ? tu.job_cost[j]
                              : double(g->n_edges + kRowCost * g->n_nodes) *
                                    est_iters(jobs[j].damping);
        const int64_t tiles = (g->n_nodes + 31) / 32;
        useful += std::max<int64_t>(1, (tiles + 4 * warps - 1) / (4 * warps));
    }
    int cap = nb_max;
    if (tu.max_blocks > 0 && tu.max_blocks < cap) cap = tu.max_blocks;
    const int nb = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(cap, useful)));
    P.nb = nb;
    if (P.claim == 2) {  // sweep: every block on every job, phase by phase
        P.nb = cap;
        P.group.assign(n_jobs, 1);
        P.items.clear();
        P.first.clear();
        return FFG_OK;
    }
    const double total = std::accumulate(cost.begin(), cost.end(), 0.0);
    const double share = total / nb;
    std::vector<int> order(n_jobs);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    P.group.assign(n_jobs, 1);
    P.items.clear();
    // Claim order: every job's ranks, consecutive, longest job first.
    // Lists: a block may hold ranks of several multi-block jobs; every block
    // runs them in the same global order (largest job first), then its
    // one-block jobs, so a group only ever waits for blocks busy with an
    // earlier job and the first job in the order always completes.  A job's
    // ranks go to the k least loaded blocks.
    std::vector<int> small;
    std::vector<std::vector<int2>> per_block(nb);
    std::vector<double> load(nb, 0.0);
    std::vector<int> by_load(nb);
    for (int j : order) {
        const int64_t tiles = (jobs[j].g->n_nodes + 31) / 32;
        // a job above `split` shares gets about one block per `grain` shares
        int k = cost[j] > tu.split * share
                    ? static_cast<int>(std::llround(cost[j] / (tu.grain * share)))
                    : 1;
        const int64_t per_rank = int64_t(warps) * std::max(1, tu.min_tiles);
        k = static_cast<int>(std::min<int64_t>(k, std::max<int64_t>(1, tiles / per_rank)));
        k = std::min(k, nb);
        if (P.claim) {  // every job in cost order, its ranks consecutive
            P.group[j] = k;
            for (int r = 0; r < k; ++r) P.items.push_back(make_int2(j, r));
            continue;
        }
        if (k < 2) {
            small.push_back(j);
            continue;
        }
        P.group[j] = k;
        std::iota(by_load.begin(), by_load.end(), 0);
        std::stable_sort(by_load.begin(), by_load.end(),
                         [&](int a, int b) { return load[a] < load[b]; });
        // the k least loaded blocks start together: they all wait for the
        // most loaded of them
        const double start = load[by_load[k - 1]];
        for (int r = 0; r < k; ++r) {
            per_block[by_load[r]].push_back(make_int2(j, r));
            load[by_load[r]] = start + cost[j] / k;
        }
    }
    P.first.clear();
    if (P.claim) return FFG_OK;
    // per-block lists: one-block jobs, longest first, onto the least loaded block
    using Slot = std::pair<double, int>;
    std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
    for (int b = 0; b < nb; ++b) heap.push({load[b], b});
    for (int j : small) {
        Slot sl = heap.top();
        heap.pop();
        per_block[sl.second].push_back(make_int2(j, 0));
        sl.first += cost[j];
        heap.push(sl);
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
    int *queue;
    int *first;
    int2 *items;
    PrCtl *ctl;
    SweepCtl *sweep_ctl;        // sweep schedule: grid barrier and failure flag
    SweepRange *sweep_ranges;   // ... each block's share of a phase, by parity
    int *sweep_ctr;             // ... units claimed from each share, by parity
    int32_t *cnt;    // per tile of every graph
    uint2 *tinfo;    // per tile of every graph
    int64_t *tpre;   // its prefix sums
    int64_t *scan;   // scan scratch (tiles)
    int32_t *aflag;  // per row of every graph: has in-edges
    int64_t *apre;   // its prefix sums
    int64_t *ascan;  // scan scratch (rows)
    int64_t total_rows;
    size_t bytes;
};

// Workspace of a plan: tables, then per job ctl / w buffers, then
// per distinct graph the layout and tile metadata.  host_jobs / host_graphs
// (if non-NULL) receive the device pointers of every job and graph.
BatchWs carve_batch(void *base, const ffg_pr_job *jobs, int n_jobs, ffg_prec prec,
                    const PlanHost &P, int cap, std::vector<JobDev> *host_jobs,
                    std::vector<GraphDev> *host_graphs) {
    Carver c(base);
    BatchWs w;
    w.jobs = c.take<JobDev>(n_jobs);
    w.graphs = c.take<GraphDev>(P.graphs.size());
    // plan tables sized for any tuning: a job has at most one item per block
    w.queue = c.take<int>(1);
    w.first = c.take<int>(size_t(cap) + 1);
    w.items = c.take<int2>(size_t(n_jobs) * cap);
    w.ctl = c.take<PrCtl>(n_jobs);
    w.sweep_ctl = c.take<SweepCtl>(1);
    w.sweep_ranges = c.take<SweepRange>(size_t(2) * cap);
    w.sweep_ctr = c.take<int>(size_t(2) * cap);
    int64_t total_tiles = 0;
    for (const ffg_graph *g : P.graphs) total_tiles += (g->n_nodes + 31) / 32;
    // per-tile descriptor counts of all graphs in one array, scanned at once
    w.cnt = c.take<int32_t>(size_t(total_tiles));
    w.tinfo = c.take<uint2>(size_t(total_tiles));
    w.tpre = c.take<int64_t>(size_t(total_tiles) + 1);
    w.scan = c.take<int64_t>(size_t(scan_scratch_elems(total_tiles)));
    int64_t total_rows = 0;
    for (const ffg_graph *g : P.graphs) total_rows += g->n_nodes;
    w.total_rows = total_rows;
    w.aflag = c.take<int32_t>(size_t(total_rows));
    w.apre = c.take<int64_t>(size_t(total_rows) + 1);
    w.ascan = c.take<int64_t>(size_t(scan_scratch_elems(total_rows)));
    std::vector<GraphDev> gd(P.graphs.size());
    int64_t tile0 = 0, row0 = 0;
    for (size_t k = 0; k < P.graphs.size(); ++k) {
        const ffg_graph *g = P.graphs[k];
        gd[k].in_ptr = g->in_ptr;
        gd[k].in_idx = g->in_idx;
        gd[k].desc = c.take<uint2>(size_t(desc_capacity(g->n_nodes, g->n_edges)));
        gd[k].cnt = w.cnt + tile0;
        gd[k].tinfo = w.tinfo + tile0;
        gd[k].perm = c.take<int32_t>(size_t(g->n_nodes));
        gd[k].aflag = w.aflag + row0;
        gd[k].apre = w.apre + row0;
        gd[k].n = g->n_nodes;
        gd[k].e = g->n_edges;
        gd[k].tile0 = tile0;
        gd[k].row0 = row0;
        tile0 += (g->n_nodes + 31) / 32;
        row0 += g->n_nodes;
    }
    std::vector<JobDev> jd(n_jobs);
    for (int j = 0; j < n_jobs; ++j) {
        const ffg_graph *g = jobs[j].g;
        const GraphDev &G = gd[P.graph_of_job[j]];
        JobDev &J = jd[j];
        J.outdeg = g->outdeg;
        J.desc = G.desc;
        J.tinfo = G.tinfo;
        J.perm = G.perm;
        J.apre = G.apre;
        J.tpre = w.tpre + G.tile0;
        J.ranks = jobs[j].ranks;
        J.w0 = c.take<char>(size_t(g->n_nodes) * w_bytes(prec));
        J.w1 = c.take<char>(size_t(g->n_nodes) * w_bytes(prec));
        J.rinv = prec == FFG_F64 ? c.take<double>(size_t(g->n_nodes)) : nullptr;
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

bool batch_width_ok(int warps) {
    return warps == kWarpsBatch || warps == kWarpsBatchWide || warps == kWarpsSingle;
}

// co-resident blocks per SM of both forms of the batch kernel
template <typename T, int W>
ffg_status batch_per_sm(int *per_sm, int *sms) {
    int a = 0, b = 0;
    FFG_TRY((kernel_config<W>((const void *)k_pagerank_batch<T, W>, &a, sms)));
    FFG_TRY((kernel_config<W>((const void *)k_pagerank_batch_p<T, W>, &b, sms)));
    *per_sm = std::min(a, b);
    return FFG_OK;
}

template <int W>
ffg_status batch_blocks_w(ffg_prec prec, int *per_sm, int *sms) {
    if (prec == FFG_F64) {
        int a = 0, b = 0;
        FFG_TRY((batch_per_sm<double, W>(&a, sms)));
        FFG_TRY((batch_per_sm<F64x, W>(&b, sms)));
        *per_sm = std::min(a, b);
        return FFG_OK;
    }
    return batch_per_sm<float, W>(per_sm, sms);
}

// co-resident blocks of the batch kernel with `warps` warps per block
ffg_status batch_blocks(ffg_prec prec, int warps, int *nb_max) {
    int per_sm = 0, sms = 0;
    if (warps == kWarpsBatch) FFG_TRY(batch_blocks_w<kWarpsBatch>(prec, &per_sm, &sms));
    else if (warps == kWarpsBatchWide) FFG_TRY(batch_blocks_w<kWarpsBatchWide>(prec, &per_sm, &sms));
    else FFG_TRY(batch_blocks_w<kWarpsSingle>(prec, &per_sm, &sms));
    *nb_max = std::min(kMaxBlocks, sms * per_sm);
    return FFG_OK;
}

// plan tables are sized for the largest of the grids, so that the
// workspace does not depend on the tuning
ffg_status batch_cap(ffg_prec prec, int *cap) {
    int a = 0, b = 0, c = 0;
    FFG_TRY(batch_blocks(prec, kWarpsBatch, &a));
    FFG_TRY(batch_blocks(prec, kWarpsBatchWide, &b));
    FFG_TRY(batch_blocks(prec, kWarpsSingle, &c));
    *cap = std::max(a, std::max(b, c));
    return FFG_OK;
}

// the batch kernel for the plan's precision and storage form of w; with the
// job table in its parameters when the plan carries it
template <int W>
ffg_status launch_batch(ffg_prec prec, bool fx, const BatchParams *P, const JobDev *jobs,
                        const int2 *items, const int *first, int *queue, int ni, int nb,
                        cudaStream_t stream) {
    if (P) {
        if (prec == FFG_F32) return launch_pr_param<float, W>(*P, nb, stream);
        if (fx) return launch_pr_param<F64x, W>(*P, nb, stream);
        return launch_pr_param<double, W>(*P, nb, stream);
    }
    if (prec == FFG_F32) return launch_pr<float, W>(jobs, items, first, queue, ni, nb, stream);
    if (fx) return launch_pr<F64x, W>(jobs, items, first, queue, ni, nb, stream);
    return launch_pr<double, W>(jobs, items, first, queue, ni, nb, stream);
}

}  // namespace
}  // namespace ffg

// per-block lists; a job above 5 % of a block's share gets about one block per
// 0.5 % of a share; the block width follows the size of the job table
// (0.05 / 0.005 was the best or close to it on both the 234-space batch and
// the 512-solve sweep)
const ffg_pr_tuning kDefaultTuning = {0.05, 0.005, 0, 0, 0, 0, 0, 0, nullptr};

extern "C" size_t pagerank_batch_workspace_bytes(const ffg_pr_job *jobs, int32_t n_jobs,
                                                 ffg_prec prec) {
    clear_error();
    if (!jobs || n_jobs < 1 || (prec != FFG_F64 && prec != FFG_F32)) return 0;
    int cap = 0, nb_max = 0;
    if (batch_cap(prec, &cap) != FFG_OK || batch_blocks(prec, kWarpsSingle, &nb_max) != FFG_OK)
        return 0;
    PlanHost P;
    if (make_plan(jobs, n_jobs, nb_max, kWarpsSingle, kDefaultTuning, P) != FFG_OK) return 0;
    return carve_batch(nullptr, jobs, n_jobs, prec, P, cap, nullptr, nullptr)
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
    // width 0: 24 warps when the job table travels in the kernel's parameters
    // (no spills), else the 16-warp form with room for the job's pointers
    const int warps = tu.block_warps          ? tu.block_warps
                      : n_jobs <= kParamJobs ? kWarpsSingle
                                             : kWarpsBatchWide;
    if (!(tu.split > 0.0) || !(tu.grain > 0.0) || tu.max_blocks < 0 || !batch_width_ok(warps) ||
        tu.claim < 0 || tu.claim > 2 || (tu.claim == 2 && warps == kWarpsBatch) ||
        tu.fp64_form < 0 || tu.fp64_form > 2 || tu.min_tiles < 0 || tu.min_tiles > (1 << 20))
        return set_error("tuning: split and grain must be > 0, max_blocks >= 0, block_warps "
                         "0, %d, %d or %d, claim 0, 1 or 2 (2 with %d or %d warps), fp64_form "
                         "0, 1 or 2, min_tiles 0..2^20",
                         kWarpsBatch, kWarpsBatchWide, kWarpsSingle, kWarpsBatchWide,
                         kWarpsSingle),
               FFG_ERR_INVALID_ARG;
    if (tu.job_cost)
        for (int j = 0; j < n_jobs; ++j)
            if (!(tu.job_cost[j] > 0.0 && tu.job_cost[j] < HUGE_VAL))
                return set_error("tuning: job_cost[%d] must be positive and finite", j),
                       FFG_ERR_INVALID_ARG;
    int cap = 0, nb_max = 0;
    FFG_TRY(batch_cap(prec, &cap));
    FFG_TRY(batch_blocks(prec, warps, &nb_max));
    if (tu.claim == 2) {  // the sweep keeps every job's state in shared memory
        int dev = 0, optin = 0;
        FFG_TRY(check_cuda(cudaGetDevice(&dev), "cudaGetDevice"));
        FFG_TRY(check_cuda(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                                  dev), "attr"));
        const size_t need = warps == kWarpsBatchWide ? sweep_smem_bytes<kWarpsBatchWide>(n_jobs)
                                                     : sweep_smem_bytes<kWarpsSingle>(n_jobs);
        if (need > size_t(optin))
            return set_error("tuning: %d jobs are too many for the sweep order", n_jobs),
                   FFG_ERR_INVALID_ARG;
    }
    PlanHost P;
    FFG_TRY(make_plan(jobs, n_jobs, nb_max, warps, tu, P));
    std::vector<JobDev> jd;
    std::vector<GraphDev> gd;
    BatchWs w = carve_batch(workspace, jobs, n_jobs, prec, P, cap, &jd, &gd);
    if (ws_bytes < w.bytes)
        return set_error("workspace %zu bytes, need %zu", ws_bytes, w.bytes), FFG_ERR_NO_MEMORY;
    if (P.nb > nb_max || P.items.size() > size_t(n_jobs) * cap)
        return set_error("internal: plan exceeds its tables"), FFG_ERR_INVALID_ARG;
    FFG_TRY(check_cuda(cudaMemcpyAsync(w.jobs, jd.data(), sizeof(JobDev) * jd.size(),
                                       cudaMemcpyHostToDevice, stream), "upload jobs"));
    FFG_TRY(check_cuda(cudaMemcpyAsync(w.graphs, gd.data(), sizeof(GraphDev) * gd.size(),
                                       cudaMemcpyHostToDevice, stream), "upload graphs"));
    if (!P.items.empty())
        FFG_TRY(check_cuda(cudaMemcpyAsync(w.items, P.items.data(), sizeof(int2) * P.items.size(),
                                           cudaMemcpyHostToDevice, stream), "upload plan"));
    if (!P.first.empty())
        FFG_TRY(check_cuda(cudaMemcpyAsync(w.first, P.first.data(), sizeof(int) * P.first.size(),
                                           cudaMemcpyHostToDevice, stream), "upload plan"));
    FFG_TRY(check_cuda(cudaStreamSynchronize(stream), "sync plan upload"));
    int64_t tiles = 0;
    for (const ffg_graph *g : P.graphs) tiles += (g->n_nodes + 31) / 32;
    plan->prec = prec;
    plan->n_jobs = n_jobs;
    plan->n_graphs = static_cast<int32_t>(P.graphs.size());
    plan->n_blocks = P.nb;
    plan->warps = P.warps;
    plan->claim = P.claim;
    int64_t n_max = 0;
    for (const ffg_graph *g : P.graphs) n_max = std::max<int64_t>(n_max, g->n_nodes);
    plan->w_form = prec == FFG_F64 && (tu.fp64_form == 1 ||
                                       (tu.fp64_form == 0 && n_max <= kFxMaxNodes))
                       ? 1
                       : 0;
    plan->n_items = static_cast<int32_t>(P.items.size());
    plan->total_tiles = tiles;
    plan->jobs = w.jobs;
    plan->graphs = w.graphs;
    plan->items = w.items;
    plan->queue = w.queue;
    plan->first = w.first;
    plan->ctl = w.ctl;
    plan->total_rows = w.total_rows;
    plan->tables[0] = w.cnt;
    plan->tables[1] = w.tpre;
    plan->tables[2] = w.scan;
    plan->tables[3] = w.aflag;
    plan->tables[4] = w.apre;
    plan->tables[5] = w.ascan;
    plan->tables[6] = w.sweep_ctl;
    plan->tables[7] = w.sweep_ranges;
    plan->tables[8] = w.sweep_ctr;
    plan->param_jobs = n_jobs <= kParamJobs ? n_jobs : 0;
    memset(plan->params, 0, sizeof(plan->params));
    if (plan->param_jobs) memcpy(plan->params, jd.data(), sizeof(JobDev) * jd.size());
    return FFG_OK;
}

namespace ffg {
namespace {

ffg_status batch_check(const ffg_pr_batch *plan) {
    if (!plan || plan->n_jobs < 1 || !plan->jobs || !plan->ctl || plan->n_blocks < 1)
        return set_error("plan is empty"), FFG_ERR_INVALID_ARG;
    if (!batch_width_ok(plan->warps))
        return set_error("plan has %d warps per block", plan->warps), FFG_ERR_INVALID_ARG;
    int nb_max = 0;
    FFG_TRY(batch_blocks(static_cast<ffg_prec>(plan->prec), plan->warps, &nb_max));
    if (plan->n_blocks > nb_max)
        return set_error("plan made for %d blocks, %d fit", plan->n_blocks, nb_max),
               FFG_ERR_INVALID_ARG;
    if (plan->param_jobs > 0 &&
        (plan->param_jobs != plan->n_jobs || plan->param_jobs > kParamJobs))
        return set_error("plan's parameter table does not match its jobs"), FFG_ERR_INVALID_ARG;
    return FFG_OK;
}

// slots, descriptors and tile costs of every distinct graph of the plan
ffg_status batch_layout(const ffg_pr_batch *plan, cudaStream_t stream) {
    int sms = 0;
    FFG_TRY(device_sms(&sms));
    const GraphDev *gr = static_cast<const GraphDev *>(plan->graphs);
    const int64_t rows = plan->total_rows;
    k_active_flags_batch<<<grid_for(rows, 256, sms), 256, 0, stream>>>(gr, plan->n_graphs, rows);
    count_launch();
    FFG_TRY(check_launch("k_active_flags_batch"));
    FFG_TRY(scan_exclusive(static_cast<const int32_t *>(plan->tables[3]),
                           static_cast<int64_t *>(plan->tables[4]), rows,
                           static_cast<int64_t *>(plan->tables[5]), stream));
    k_perm_batch<<<grid_for(rows, 256, sms), 256, 0, stream>>>(gr, plan->n_graphs, rows);
    count_launch();
    FFG_TRY(check_launch("k_perm_batch"));
    k_pr_layout_batch<<<grid_for(plan->total_tiles, kLayoutThreads / 32, sms), kLayoutThreads, 0,
                        stream>>>(gr, plan->n_graphs, plan->total_tiles);
    count_launch();
    FFG_TRY(check_launch("k_pr_layout_batch"));
    return scan_exclusive(static_cast<const int32_t *>(plan->tables[0]),
                          static_cast<int64_t *>(plan->tables[1]), plan->total_tiles,
                          static_cast<int64_t *>(plan->tables[2]), stream);
}

// the sweep kernel for the plan's precision and storage form of w
template <typename T, int W>
ffg_status launch_sweep_t(const SweepArgs &A, cudaStream_t stream) {
    const size_t smem = sweep_smem_bytes<W>(A.n_jobs);
    const void *kern = (const void *)k_pagerank_sweep<T, W>;
    FFG_TRY(check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            static_cast<int>(smem)),
                       "smem attribute"));
    int per_sm = 0;
    FFG_TRY(check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * W, smem),
                       "occupancy"));
    int sms = 0;
    FFG_TRY(device_sms(&sms));
    if (per_sm < 1 || A.nb > sms * per_sm)
        return set_error("sweep plan of %d blocks does not fit (%d per SM)", A.nb, per_sm),
               FFG_ERR_INVALID_ARG;
    SweepArgs a = A;
    void *args[] = {(void *)&a};
    FFG_TRY(check_cuda(cudaLaunchCooperativeKernel(kern, dim3(A.nb), dim3(32 * W), args, smem,
                                                   stream),
                       "k_pagerank_sweep"));
    count_launch();
    return FFG_OK;
}

template <int W>
ffg_status launch_sweep(ffg_prec prec, bool fx, const SweepArgs &A, cudaStream_t stream) {
    if (prec == FFG_F32) return launch_sweep_t<float, W>(A, stream);
    if (fx) return launch_sweep_t<F64x, W>(A, stream);
    return launch_sweep_t<double, W>(A, stream);
}

// the persistent launch over every job
ffg_status batch_solve(const ffg_pr_batch *plan, cudaStream_t stream) {
    const ffg_prec prec = static_cast<ffg_prec>(plan->prec);
    FFG_TRY(check_cuda(cudaMemsetAsync(plan->ctl, 0, sizeof(PrCtl) * plan->n_jobs, stream),
                       "memset"));
    if (plan->claim == 2) {
        SweepArgs A;
        A.jobs = static_cast<const JobDev *>(plan->jobs);
        A.ctl = static_cast<SweepCtl *>(plan->tables[6]);
        A.ranges = static_cast<SweepRange *>(plan->tables[7]);
        A.ctr = static_cast<int *>(plan->tables[8]);
        A.n_jobs = plan->n_jobs;
        A.nb = plan->n_blocks;
        FFG_TRY(check_cuda(cudaMemsetAsync(A.ctl, 0, sizeof(SweepCtl), stream), "memset"));
        FFG_TRY(check_cuda(cudaMemsetAsync(A.ranges, 0xff, sizeof(SweepRange) * 2 * A.nb, stream),
                           "memset"));
        FFG_TRY(check_cuda(cudaMemsetAsync(A.ctr, 0, sizeof(int) * 2 * A.nb, stream), "memset"));
        const bool fx = plan->w_form != 0;
        if (plan->warps == kWarpsBatchWide) return launch_sweep<kWarpsBatchWide>(prec, fx, A, stream);
        return launch_sweep<kWarpsSingle>(prec, fx, A, stream);
    }
    FFG_TRY(check_cuda(cudaMemsetAsync(plan->queue, 0, sizeof(int), stream), "memset"));
    const JobDev *jobs = static_cast<const JobDev *>(plan->jobs);
    const int2 *items = static_cast<const int2 *>(plan->items);
    const int *first = static_cast<const int *>(plan->first);
    int *queue = plan->claim ? static_cast<int *>(plan->queue) : nullptr;
    const int ni = plan->n_items, nb = plan->n_blocks;
    const bool fx = plan->w_form != 0;  // FP64 w stored in fixed point
    // batches of at most kParamJobs jobs pass their job table as parameters
    std::unique_ptr<BatchParams> params;
    if (plan->param_jobs > 0) {
        params.reset(new BatchParams());
        params->items = items;
        params->first = first;
        params->queue = queue;
        params->n_items = ni;
        memcpy(params->jobs, plan->params, sizeof(JobDev) * size_t(plan->param_jobs));
    }
    const BatchParams *P = params.get();
    if (plan->warps == kWarpsBatch)
        return launch_batch<kWarpsBatch>(prec, fx, P, jobs, items, first, queue, ni, nb, stream);
    if (plan->warps == kWarpsBatchWide)
        return launch_batch<kWarpsBatchWide>(prec, fx, P, jobs, items, first, queue, ni, nb,
                                             stream);
    return launch_batch<kWarpsSingle>(prec, fx, P, jobs, items, first, queue, ni, nb, stream);
}

}  // namespace
}  // namespace ffg

extern "C" ffg_status pagerank_batch_run(const ffg_pr_batch *plan, void *stream_) {
    clear_error();
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    FFG_TRY(batch_check(plan));
    FFG_TRY(batch_layout(plan, stream));
    return batch_solve(plan, stream);
}

extern "C" ffg_status pagerank_batch_prepare(const ffg_pr_batch *plan, void *stream_) {
    clear_error();
    FFG_TRY(batch_check(plan));
    return batch_layout(plan, static_cast<cudaStream_t>(stream_));
}

extern "C" ffg_status pagerank_batch_solve(const ffg_pr_batch *plan, void *stream_) {
    clear_error();
    FFG_TRY(batch_check(plan));
    return batch_solve(plan, static_cast<cudaStream_t>(stream_));
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

extern "C" ffg_status pagerank_batch_times(const ffg_pr_batch *plan, double *block_seconds_out,
                                           void *stream_) {
    clear_error();
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (!plan || plan->n_jobs < 1 || !plan->ctl || !block_seconds_out)
        return set_error("plan is empty or block_seconds_out NULL"), FFG_ERR_INVALID_ARG;
    std::vector<PrCtl> h(plan->n_jobs);
    FFG_TRY(check_cuda(cudaMemcpyAsync(h.data(), plan->ctl, sizeof(PrCtl) * h.size(),
                                       cudaMemcpyDeviceToHost, stream), "read batch times"));
    FFG_TRY(check_cuda(cudaStreamSynchronize(stream), "sync batch times"));
    for (int j = 0; j < plan->n_jobs; ++j) block_seconds_out[j] = 1e-9 * double(h[j].busy_ns);
    return FFG_OK;
}

namespace ffg {
FFG_CHECK_READER(check_read_pagerank)
}  // namespace ffg
