// reduce.cuh -- block-level FP64 reductions shared by the reduction kernels
// (warp shuffles, then a shared-memory tree of the warp results; results in
// thread 0).  Blocks of RT threads.
#pragma once
#include <cuda_runtime.h>

namespace aafwi {

constexpr int RT = 256;  // threads per reduction block

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    v = threadIdx.x < RT / 32 ? sh[threadIdx.x] : 0.0;
    if (w == 0) v = warp_sum(v);
    return v;
}

// Block-wide maximum of non-negative values; result valid in thread 0.
__device__ __forceinline__ double block_max(double v, double *sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_max(v);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    v = threadIdx.x < RT / 32 ? sh[threadIdx.x] : 0.0;
    if (w == 0) v = warp_max(v);
    return v;
}

}  // namespace aafwi
