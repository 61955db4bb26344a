// Warp and block exclusive scans of one int per thread, the building blocks of
// the three-phase device scans (block sums, a scan of the block sums, the
// block-local scans with their offsets) used for cell offsets and pair-record
// offsets.
#pragma once

namespace espp {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// block-wide exclusive scan of one int per thread; returns the block total
__device__ __forceinline__ int block_excl_scan(int v, int* excl_out) {
    __shared__ int wsum[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = warp_incl_scan(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        int t = lane < SCAN_THREADS / 32 ? wsum[lane] : 0;
        t = warp_incl_scan(t);
        if (lane < SCAN_THREADS / 32) wsum[lane] = t;
    }
    __syncthreads();
    const int base = w > 0 ? wsum[w - 1] : 0;
    *excl_out = base + inc - v;
    const int total = wsum[SCAN_THREADS / 32 - 1];
    __syncthreads();
    return total;
}

}  // namespace espp
