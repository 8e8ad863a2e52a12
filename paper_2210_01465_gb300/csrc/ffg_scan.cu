// ffg_scan.cu -- deterministic device-wide exclusive scan of int32 counts into
// int64 offsets (node numbering, CSR row pointers).  Three launches: tile
// sums, one block scanning the tile sums, tile-local scans plus offsets.
#include "ffg_internal.cuh"

namespace ffg {

namespace {

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// exclusive scan over the block; returns this thread's offset, *total = sum
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *total) {
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t block_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    int64_t incl = warp_incl_scan(v);
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < nwarps ? warp_sums[lane] : 0;
        int64_t wi = warp_incl_scan(w);
        if (lane < nwarps) warp_sums[lane] = wi - w;
        if (lane == 31) block_total = wi;
    }
    __syncthreads();
    int64_t r = warp_sums[warp] + incl - v;
    *total = block_total;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int32_t *__restrict__ in,
                                                               int64_t n,
                                                               int64_t *__restrict__ sums) {
    const int64_t base = int64_t(blockIdx.x) * kScanTile;
    int64_t s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + int64_t(k) * kScanThreads + threadIdx.x;
        if (i < n) s += in[i];
    }
    int64_t total;
    block_excl_scan(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// one block: exclusive scan of sums[0..nb) in place, sums[nb] = total
__global__ void __launch_bounds__(1024) k_scan_top(int64_t *sums, int64_t nb) {
    int64_t carry = 0;
    for (int64_t base = 0; base < nb; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < nb ? sums[i] : 0;
        int64_t total;
        int64_t ex = block_excl_scan(v, &total);
        if (i < nb) sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const int32_t *__restrict__ in,
                                                             int64_t n,
                                                             const int64_t *__restrict__ sums,
                                                             int64_t nb,
                                                             int64_t *__restrict__ out) {
    __shared__ int32_t tile[kScanTile];
    const int64_t base = int64_t(blockIdx.x) * kScanTile;
    // coalesced load into shared memory, then each thread scans 8 consecutive
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + int64_t(k) * kScanThreads + threadIdx.x;
        tile[k * kScanThreads + threadIdx.x] = i < n ? in[i] : 0;
    }
    __syncthreads();
    int32_t v[kScanItems];
    int64_t s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = tile[threadIdx.x * kScanItems + k];
        s += v[k];
    }
    int64_t total;
    int64_t off = block_excl_scan(s, &total) + sums[blockIdx.x];
    int64_t res[kScanItems];
    for (int k = 0; k < kScanItems; ++k) {
        res[k] = off;
        off += v[k];
    }
    // write back through shared memory for coalesced stores
    __shared__ int64_t otile[kScanTile];
    for (int k = 0; k < kScanItems; ++k) otile[threadIdx.x * kScanItems + k] = res[k];
    __syncthreads();
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + int64_t(k) * kScanThreads + threadIdx.x;
        if (i < n) out[i] = otile[k * kScanThreads + threadIdx.x];
    }
    if (blockIdx.x == nb - 1 && threadIdx.x == 0) out[n] = sums[nb];
}

}  // namespace

ffg_status scan_exclusive(const int32_t *in, int64_t *out, int64_t n, int64_t *scratch,
                          cudaStream_t stream) {
    if (n <= 0) {
        FFG_TRY(check_cuda(cudaMemsetAsync(out, 0, sizeof(int64_t), stream), "scan memset"));
        return FFG_OK;
    }
    const int64_t nb = scan_blocks(n);
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, stream>>>(in, n, scratch);
    k_scan_top<<<1, 1024, 0, stream>>>(scratch, nb);
    k_scan_down<<<(unsigned)nb, kScanThreads, 0, stream>>>(in, n, scratch, nb, out);
    count_launch(3);
    return check_launch("scan");
}

}  // namespace ffg
