// Deterministic block / grid reductions (warp shuffles, then the last-block
// pattern: every block stores one partial, the last block to finish sums the
// partials in a fixed order -- no atomics on data, no spinning).
#pragma once
#include "common.cuh"

namespace jfnk {

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block of one double per warp-summed value.  All threads must
// call it.  `sm` holds >= 32 doubles.  Result valid in thread 0.
template <typename TA>
__device__ __forceinline__ double block_sum(TA v, double* sm) {
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    TA w = warp_sum(v);
    if ((tid & 31) == 0) sm[tid >> 5] = (double)w;
    __syncthreads();
    double t = 0.0;
    if (tid < 32) {
        t = (tid < (nt + 31) / 32) ? sm[tid] : 0.0;
        t = warp_sum(t);
    }
    __syncthreads();
    return t;
}

// Last-block completion over a segment of nb CTAs (bid = this CTA's index in
// it).  Thread 0 of every block passes its block sum; returns true in every
// thread of the last block of the segment, with the total in *total (thread
// 0).  The completion counter is reset by the last block.
__device__ __forceinline__ bool grid_sum_last_seg(double blocksum, double* partials, unsigned int* counter,
                                                  double* total, double* sm, unsigned int bid, unsigned int nb) {
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nt = blockDim.x * blockDim.y * blockDim.z;
    if (nb == 1) {  // the only block: no partials, no completion counter
        if (tid == 0) *total = blocksum;
        return true;
    }
    __shared__ int s_last;
    if (tid == 0) {
        partials[bid] = blocksum;
        __threadfence();
        unsigned int prev = atomicAdd(counter, 1u);
        s_last = (prev == nb - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double s = 0.0;
    for (unsigned int i = tid; i < nb; i += nt) s += __ldcg(&partials[i]);
    s = block_sum(s, sm);
    if (tid == 0) {
        *total = s;
        *counter = 0u;
    }
    return true;
}

// The whole grid as one segment.
__device__ __forceinline__ bool grid_sum_last(double blocksum, double* partials, unsigned int* counter,
                                              double* total, double* sm) {
    return grid_sum_last_seg(blocksum, partials, counter, total, sm,
                             blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z),
                             gridDim.x * gridDim.y * gridDim.z);
}

}  // namespace jfnk
