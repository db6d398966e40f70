// Device helpers shared by the CUDA translation units of the library: CTA
// sums in a fixed order and the last-CTA reduction of per-CTA partial sums
// (the classic threadfence reduction: no CTA waits for another).
#pragma once

#include <cuda_runtime.h>

#include "ht_internal.cuh"

namespace ht {

// Sum over the CTA (1D, 2D or 3D blocks whose size is a multiple of 32);
// the result is valid in the thread with linear index 0.
// Block sum of per-thread partials of a T-typed kernel: the warp stage runs
// in T (for FP32 kernels this keeps the shuffles and adds off the FP64 pipe,
// which GB300 runs at 1/64 of the FP32 rate), the per-warp results are
// combined in FP64 by block_sum.  Valid in thread 0; fixed order.
template <typename T>
__device__ __forceinline__ double block_sum_t(T v);

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int lane = tid & 31, wid = tid >> 5;
    __syncthreads();
    if (lane == 0) ws[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x * blockDim.y * blockDim.z + 31) >> 5;
    v = (tid < nw) ? ws[lane] : 0.0;
    if (wid == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

template <typename T>
__device__ __forceinline__ double block_sum_t(T v) {
    if constexpr (sizeof(T) == 8) return block_sum((double)v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __shared__ double wsum[32];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int lane = tid & 31, wid = tid >> 5;
    __syncthreads();
    if (lane == 0) wsum[wid] = (double)v;
    __syncthreads();
    double d = 0.0;
    if (tid == 0) {
        const int nw = (blockDim.x * blockDim.y * blockDim.z + 31) >> 5;
        for (int w = 0; w < nw; ++w) d += wsum[w];
    }
    return d;
}

// thread 0 publishes the CTA's partial sums and takes a ticket; the result is
// true in every thread of the CTA that finished last
__device__ __forceinline__ bool publish_and_ticket(Scal* s, double* part_slot, const double* vals, int nv,
                                                   int stride, unsigned nblk) {
    __shared__ bool last;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const unsigned blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    if (tid == 0) {
        for (int k = 0; k < nv; ++k) part_slot[(size_t)k * stride + blk] = vals[k];
        __threadfence();
        last = atomicAdd(&s->ticket, 1u) == nblk - 1;
    }
    __syncthreads();
    return last;
}

// sum of part[0..n) in a fixed order (valid in thread 0); reads bypass L1
__device__ __forceinline__ double last_cta_sum(const double* part, int n) {
    const int tid = threadIdx.x + blockDim.x * threadIdx.y, nt = blockDim.x * blockDim.y;
    double a = 0.0;
    for (int i = tid; i < n; i += nt) a += __ldcg(part + i);
    return block_sum(a);
}

}  // namespace ht
