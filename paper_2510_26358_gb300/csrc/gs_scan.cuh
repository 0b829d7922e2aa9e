// Block-wide sums and exclusive scans of one 32-bit value per thread, for
// the compaction kernels (lifecycle, voxel insertion, partitions).  NT is
// the block size (a multiple of 32); sm holds NT / 32 values.  Every thread
// of the block must call them (they synchronise).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gs {

template <int NT>
__device__ __forceinline__ uint32_t block_sum_u32(uint32_t v, uint32_t *sm) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[w] = v;
    __syncthreads();
    uint32_t t = 0;
    for (int i = 0; i < NT / 32; ++i) t += sm[i];
    return t;
}

// exclusive prefix of v over the block; `total` receives the block sum
template <int NT>
__device__ __forceinline__ uint32_t block_scan_u32(uint32_t v, uint32_t *sm, uint32_t &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) sm[w] = x;
    __syncthreads();
    uint32_t wpre = 0;
    total = 0;
    for (int i = 0; i < NT / 32; ++i) {
        if (i < w) wpre += sm[i];
        total += sm[i];
    }
    return wpre + x - v;
}

}  // namespace gs
