// Device helpers shared by the operator kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fem_internal.h"

namespace fem {

// Elements per block for a slab of q x q threads per element: enough
// threads to keep several warps per block, bounded by the shared-memory
// budget (bytes per element given).
__host__ __device__ constexpr int pick_epb(int q, int smem_per_elem) {
    int t = 256 / (q * q);
    if (t < 1) t = 1;
    while (t > 1 && t * smem_per_elem > 96 * 1024) t--;
    return t;
}

// Rounds a count of doubles up to a multiple of 2 (16-byte alignment).
__host__ __device__ constexpr int pad2(int x) { return (x + 1) & ~1; }

// Copies `count` doubles from global to shared with all threads of the block.
__device__ __forceinline__ void block_copy(double *dst, const double *__restrict__ src, int count) {
    for (int t = threadIdx.x; t < count; t += blockDim.x) dst[t] = __ldg(src + t);
}

// Sum of v over the block (blockDim.x a multiple of 32), in a fixed order so
// that repeated runs give identical bits; the result is valid in thread 0.
// sh: at least 32 doubles of shared memory not in use by other threads.
// Every thread of the block must call it.
__device__ __forceinline__ double block_sum(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    v = (threadIdx.x < (unsigned)nw) ? sh[threadIdx.x] : 0.0;
    if (w == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// Dispatch of a functor templated on the degree N (1..15) at run time.
template <template <int> class F, typename... Args>
cudaError_t dispatch_degree(int N, Args &&...args) {
    switch (N) {
#define FEM_CASE(K) \
    case K:         \
        return F<K>::run(args...);
        FEM_CASE(1) FEM_CASE(2) FEM_CASE(3) FEM_CASE(4) FEM_CASE(5)
        FEM_CASE(6) FEM_CASE(7) FEM_CASE(8) FEM_CASE(9) FEM_CASE(10)
        FEM_CASE(11) FEM_CASE(12) FEM_CASE(13) FEM_CASE(14) FEM_CASE(15)
#undef FEM_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace fem
