// ffg_internal.cuh -- shared internals of the sm_103a FFG library: the device
// copy of a search space, its host-side validation, error reporting, the
// launch counter and workspace carving.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/ffg.h"

namespace ffg {

// ---------------------------------------------------------------------------
// diagnostics
// ---------------------------------------------------------------------------
void set_error(const char *fmt, ...);
void clear_error();
extern std::atomic<uint64_t> g_launches;
inline void count_launch(uint64_t n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// cudaGetLastError after a launch; returns FFG_ERR_CUDA with the message.
ffg_status check_launch(const char *what);
ffg_status check_cuda(cudaError_t e, const char *what);

#define FFG_TRY(expr)                           \
    do {                                        \
        ffg_status _s = (expr);                 \
        if (_s != FFG_OK) return _s;            \
    } while (0)

// ---------------------------------------------------------------------------
// bounds-checked builds (-DFFG_CHECKED)
// Every index a kernel derives from caller data (a CSR entry, a descriptor
// offset, a row pointer) is checked before the access it guards; a failed
// check skips the access and records its site code in a word of the
// translation unit, which ffg_checked_failures() reads.  Normal builds
// compile the checks away (FFG_CHECK is `true`).
// ---------------------------------------------------------------------------
#ifdef FFG_CHECKED
static __device__ unsigned long long g_check_code;   // first failed site, 0 if none
static __device__ unsigned long long g_check_count;  // failed checks
__device__ __forceinline__ bool ffg_check(bool ok, unsigned code) {
    if (!ok) {
        atomicCAS(&g_check_code, 0ULL, static_cast<unsigned long long>(code));
        atomicAdd(&g_check_count, 1ULL);
    }
    return ok;
}
#define FFG_CHECK(cond, code) ffg::ffg_check((cond), (code))
// this translation unit's words (host side; reset clears them)
static inline void check_read_tu(unsigned long long *code, unsigned long long *count,
                                 bool reset) {
    cudaMemcpyFromSymbol(code, g_check_code, sizeof(*code));
    cudaMemcpyFromSymbol(count, g_check_count, sizeof(*count));
    if (reset) {
        const unsigned long long z = 0;
        cudaMemcpyToSymbol(g_check_code, &z, sizeof(z));
        cudaMemcpyToSymbol(g_check_count, &z, sizeof(z));
    }
}
#define FFG_CHECK_READER(name)                                                         \
    void name(unsigned long long *code, unsigned long long *count, bool reset) {       \
        check_read_tu(code, count, reset);                                            \
    }
#else
#define FFG_CHECK(cond, code) true
#define FFG_CHECK_READER(name)                                                         \
    void name(unsigned long long *code, unsigned long long *count, bool) {             \
        *code = 0;                                                                    \
        *count = 0;                                                                   \
    }
#endif
// the readers of the translation units with checks
void check_read_build(unsigned long long *, unsigned long long *, bool);
void check_read_pagerank(unsigned long long *, unsigned long long *, bool);
void check_read_dag(unsigned long long *, unsigned long long *, bool);
void check_read_walk(unsigned long long *, unsigned long long *, bool);
void check_read_centrality(unsigned long long *, unsigned long long *, bool);

// ---------------------------------------------------------------------------
// device copy of a search space (passed to kernels by value)
// ---------------------------------------------------------------------------
struct DevClause {
    int32_t kind;
    uint32_t mask_a, mask_b;
    int32_t pad;
    int64_t bound;
};

struct DevSpace {
    int32_t n_params, n_clauses, n_values, pad;
    int64_t n_raw;
    int32_t radix[FFG_MAX_PARAMS];
    int32_t voff[FFG_MAX_PARAMS];
    int64_t stride[FFG_MAX_PARAMS];
    DevClause clause[FFG_MAX_CONSTRAINTS];
    int64_t values[FFG_MAX_VALUES];
};

// Validates `s` and fills `d` (strides, offsets, overflow checks).
ffg_status make_dev_space(const ffg_space *s, DevSpace *d);

// ---------------------------------------------------------------------------
// workspace carving: consecutive 256-byte aligned slices
// ---------------------------------------------------------------------------
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base(static_cast<char *>(b)) {}
    template <typename T>
    T *take(size_t count) {
        size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += bytes;
        return p;
    }
};

inline bool aligned256(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 255) == 0; }

// ---------------------------------------------------------------------------
// device-wide exclusive scan of non-negative int32 counts into int64 offsets:
// out[0..n] with out[n] = total.  `scratch` needs scan_scratch_elems(n) int64.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int64_t kScanTile = int64_t(kScanThreads) * kScanItems;
inline int64_t scan_blocks(int64_t n) { return (n + kScanTile - 1) / kScanTile; }
inline int64_t scan_scratch_elems(int64_t n) { return scan_blocks(n) + 2; }
ffg_status scan_exclusive(const int32_t *in, int64_t *out, int64_t n, int64_t *scratch,
                          cudaStream_t stream);

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
// failed configurations (fitness not below the threshold, NaN included)
// compare as +infinity
__device__ __forceinline__ double fit_key(double f, double fail_thr) {
    return (f < fail_thr) ? f : __longlong_as_double(0x7ff0000000000000LL);
}

// order-preserving map of a double onto uint64 (for atomicMin)
__device__ __forceinline__ unsigned long long ordered_bits(double x) {
    unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    return (b & 0x8000000000000000ULL) ? ~b : (b | 0x8000000000000000ULL);
}
__host__ __device__ inline double from_ordered_bits(unsigned long long b) {
    unsigned long long r = (b & 0x8000000000000000ULL) ? (b & 0x7fffffffffffffffULL) : ~b;
    double d;
    memcpy(&d, &r, sizeof(d));
    return d;
}

}  // namespace ffg
