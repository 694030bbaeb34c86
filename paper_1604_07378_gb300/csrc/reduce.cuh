// Deterministic block and grid reductions.  A grid reduction writes one
// partial per block; the last block to arrive (an arrival ticket, the only
// atomic used) sums the partials in a fixed order, so results do not depend
// on block scheduling.
#pragma once

#include "common.cuh"

namespace hqn {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename R>
__device__ __forceinline__ R warp_sum_r(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of NV doubles over the block; the result is valid in thread 0.
template <int BS, int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
    __shared__ double sh[NV][BS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k][warp] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = lane < BS / 32 ? sh[k][lane] : 0.0;
            v[k] = warp_sum(t);
        }
    }
    __syncthreads();
}

// Sum of NV values over the block, first within each warp in the working
// precision R, then across the warps in float64; the result (float64) is
// valid in thread 0.  Used for the two-loop's inner products, whose terms are
// R-precision products anyway; with R = double it equals block_sum.
template <int BS, int NV, typename R>
__device__ __forceinline__ void block_sum_mixed(const R (&v)[NV], double (&out)[NV]) {
    __shared__ double sh[NV][BS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const R t = warp_sum_r(v[k]);
        if (lane == 0) sh[k][warp] = (double)t;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) out[k] = warp_sum(lane < BS / 32 ? sh[k][lane] : 0.0);
    }
    __syncthreads();
}

// Thread 0 publishes the block's partials (part[k * stride + blockIdx.x]) and
// takes an arrival ticket.  Returns true in every thread of the last block.
template <int NV>
__device__ __forceinline__ bool publish_and_arrive(const double (&v)[NV], double *part, int stride,
                                                   unsigned int *ticket) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) part[k * stride + blockIdx.x] = v[k];
        __threadfence();
        const unsigned int t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    return last;
}

// In the last block: fixed-order sums of NV partial arrays of length n.
// Result valid in thread 0; thread 0 also re-arms the ticket.
template <int BS, int NV>
__device__ __forceinline__ void sum_partials(const double *part, int stride, int n, double (&out)[NV],
                                             unsigned int *ticket) {
    __threadfence();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < n; i += BS) acc += __ldcg(part + k * stride + i);
        out[k] = acc;
    }
    block_sum<BS, NV>(out);
    if (threadIdx.x == 0) *ticket = 0u;
}

}  // namespace hqn
