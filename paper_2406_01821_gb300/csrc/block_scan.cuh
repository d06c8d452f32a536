// Block-wide exclusive prefix sum with warp shuffles.
#pragma once
#include <cuda_runtime.h>

namespace rs {

// Exclusive prefix of one int per thread over the block (blockDim.x a multiple of 32, at most
// 1024; every thread of the block calls it); the block's total goes to *total.
__device__ __forceinline__ int block_exclusive_scan(int v, int *total)
{
    __shared__ int warp_sums[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int t = lane < nw ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_sums[lane] = t;
    }
    __syncthreads();
    const int excl = x - v + (warp ? warp_sums[warp - 1] : 0);
    *total = warp_sums[nw - 1];
    __syncthreads();                  // warp_sums is reused by the next call
    return excl;
}

// In-place exclusive prefix of n counters in shared memory by the whole block (n a multiple of
// blockDim.x; every thread calls it).
__device__ __forceinline__ void block_exclusive_scan_array(int *h, int n)
{
    const int per = n / blockDim.x, base = threadIdx.x * per;
    int local = 0;
    for (int i = 0; i < per; ++i) local += h[base + i];
    int total = 0;
    int run = block_exclusive_scan(local, &total);
    for (int i = 0; i < per; ++i) {
        const int c = h[base + i];
        h[base + i] = run;
        run += c;
    }
    __syncthreads();
}

}  // namespace rs
