// Deterministic block and grid reductions.  A grid reduction writes one
// partial per block; the last block to arrive (an arrival ticket, the only
// atomic used) sums the partials in a fixed order, so results do not depend
// on block scheduling.
//
// GB300 issues float64 arithmetic at a small fraction of its float32 rate, so
// sums that must be float64-accurate (energies, rho = s^T t) accumulate in
// float-float pairs inside warps and blocks -- a float hi plus a float lo
// carrying its rounding error (Knuth's TwoSum; exact products by FMA, Dekker)
// -- and become doubles only for the per-block partials.  Sums that may be
// float32 (the other inner products of Alg. 2) use float32 up to the block
// partial.  The final sum over the partials is float64, one warp per value.
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

// ---- float-float accumulators

struct FF {
    float hi, lo;
};

// s + e = a + b exactly (Knuth's TwoSum, no ordering condition).
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return FF{s, e};
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
    const FF s = ff_two_sum(a.hi, b.hi);
    const float e = s.lo + (a.lo + b.lo);
    const float h = s.hi + e;
    return FF{h, e - (h - s.hi)};
}

// a * b exactly as hi + lo (the FMA computes the rounding error of the product).
__device__ __forceinline__ FF ff_prod(float a, float b) {
    const float p = a * b;
    return FF{p, fmaf(a, b, -p)};
}

__device__ __forceinline__ double ff_to_double(FF a) { return (double)a.hi + (double)a.lo; }

// Accumulator of float64-accurate sums in working precision R: float-float
// for float, double for double.
template <typename R> struct ExactAcc;
template <> struct ExactAcc<float> {
    using T = FF;
    __device__ static T zero() { return FF{0.f, 0.f}; }
    __device__ static T add(T a, float x) { return ff_add(a, FF{x, 0.f}); }
    __device__ static T add_prod(T a, float x, float y) { return ff_add(a, ff_prod(x, y)); }
    __device__ static T combine(T a, T b) { return ff_add(a, b); }
    __device__ static T shfl_xor(T a, int o) {
        return FF{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
    }
    __device__ static double to_double(T a) { return ff_to_double(a); }
};
template <> struct ExactAcc<double> {
    using T = double;
    __device__ static T zero() { return 0.0; }
    __device__ static T add(T a, double x) { return a + x; }
    __device__ static T add_prod(T a, double x, double y) { return fma(x, y, a); }
    __device__ static T combine(T a, T b) { return a + b; }
    __device__ static T shfl_xor(T a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
    __device__ static double to_double(T a) { return a; }
};

// ---- block sums (results valid in thread 0)

// NV float64 values, float64 throughout.
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

// NV float64-accurate sums accumulated in ExactAcc<R>.
template <int BS, int NV, typename R>
__device__ __forceinline__ void block_sum_exact(typename ExactAcc<R>::T (&v)[NV], double (&out)[NV]) {
    using A = ExactAcc<R>;
    using T = typename A::T;
    __shared__ T sh[NV][BS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        T t = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t = A::combine(t, A::shfl_xor(t, o));
        if (lane == 0) sh[k][warp] = t;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            T t = lane < BS / 32 ? sh[k][lane] : A::zero();
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t = A::combine(t, A::shfl_xor(t, o));
            out[k] = A::to_double(t);
        }
    }
    __syncthreads();
}

// NV sums in working precision R up to the block partial (R = double: float64).
template <int BS, int NV, typename R>
__device__ __forceinline__ void block_sum_r(const R (&v)[NV], double (&out)[NV]) {
    __shared__ R sh[NV][BS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const R t = warp_sum_r(v[k]);
        if (lane == 0) sh[k][warp] = t;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) out[k] = (double)warp_sum_r(lane < BS / 32 ? sh[k][lane] : R(0));
    }
    __syncthreads();
}

// ---- grid level

// part[j] + part[j + stride] + ... (indices < n), added in that order; eight
// terms are loaded before any is added, so a thread's sum costs one memory
// round trip per eight terms rather than one per term.
__device__ __forceinline__ double strided_sum(const double *part, int j, int n, int stride) {
    double acc = 0.0;
    for (int b = j; b < n; b += 8 * stride) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int bb = b + u * stride;
            v[u] = bb < n ? __ldcg(part + bb) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) acc += v[u];
    }
    return acc;
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
        __threadfence();  // release: the partials before the ticket
        const unsigned int t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
        if (last) __threadfence();  // acquire, ordered for the block by the barrier below
    }
    __syncthreads();
    return last;
}

// ---- block partials of float64-accurate sums
//
// A block partial occupies the 8 bytes of a double.  In float mode it is a
// float-float pair and the simulation's last block adds the partials in
// float-float arithmetic: GB300 issues float64 at a small fraction of the
// float32 rate, and a chain of float64 additions on the one SM that finishes
// a grid reduction was the tail of every reducing kernel.  In double mode
// partials stay doubles.  The conversions are exact (a double that is the
// sum of a float-float pair splits back into the same pair).
template <typename R> struct Part;
template <> struct Part<float> {
    using T = FF;
    __device__ static void put(double *slot, double v) {
        const float hi = (float)v;
        const float lo = (float)(v - (double)hi);
        *reinterpret_cast<float2 *>(slot) = make_float2(hi, lo);
    }
    __device__ static T get(const double *slot) {
        const float2 f = __ldcg(reinterpret_cast<const float2 *>(slot));
        return FF{f.x, f.y};
    }
    __device__ static T zero() { return FF{0.f, 0.f}; }
    __device__ static T add(T a, T b) { return ff_add(a, b); }
    __device__ static T shfl_xor(T a, int o) {
        return FF{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
    }
    __device__ static double to_double(T a) { return ff_to_double(a); }
};
template <> struct Part<double> {
    using T = double;
    __device__ static void put(double *slot, double v) { *slot = v; }
    __device__ static T get(const double *slot) { return __ldcg(slot); }
    __device__ static T zero() { return 0.0; }
    __device__ static T add(T a, T b) { return a + b; }
    __device__ static T shfl_xor(T a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
    __device__ static double to_double(T a) { return a; }
};

template <typename R>
__device__ __forceinline__ typename Part<R>::T part_warp_sum(typename Part<R>::T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = Part<R>::add(v, Part<R>::shfl_xor(v, o));
    return v;
}

// part[j] + part[j + stride] + ... (indices < n) as Part<R> values, added in
// that order, eight loads in flight per round.
template <typename R>
__device__ __forceinline__ typename Part<R>::T part_strided_sum(const double *part, int j, int n, int stride) {
    using P = Part<R>;
    typename P::T acc = P::zero();
    for (int b = j; b < n; b += 8 * stride) {
        typename P::T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int bb = b + u * stride;
            v[u] = bb < n ? P::get(part + bb) : P::zero();
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) acc = P::add(acc, v[u]);
    }
    return acc;
}

// Fixed-order sums of NV partial arrays (value k at part[k * stride + b],
// b < n, stored by Part<R>::put) by the NW warps of a block: warp w takes the values k = w,
// w + NW, ...; a lane adds the partials b = lane, lane + 32, ... in that order
// (as strided_sum does) with the loads of all of the warp's values issued
// together, so the whole sum costs one memory round trip per 256 partials.
// Results in sh[k] (lane 0 writes them; the caller synchronises).
template <typename R, int NV, int NW>
__device__ __forceinline__ void warp_value_sums(const double *part, size_t stride, int n, double *sh) {
    using P = Part<R>;
    constexpr int PER = (NV + NW - 1) / NW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    typename P::T acc[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) acc[q] = P::zero();
    for (int b0 = lane; b0 < n; b0 += 32 * 8) {
        typename P::T v[PER][8];
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int k = warp + q * NW;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int bb = b0 + u * 32;
                v[q][u] = (k < NV && bb < n) ? P::get(part + (size_t)k * stride + bb) : P::zero();
            }
        }
#pragma unroll
        for (int q = 0; q < PER; ++q)
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[q] = P::add(acc[q], v[q][u]);
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int k = warp + q * NW;
        if (k < NV) {
            const typename P::T a = part_warp_sum<R>(acc[q]);
            if (lane == 0) sh[k] = P::to_double(a);
        }
    }
}

// In the last block: fixed-order float64 sums of NV partial arrays of length
// n, one warp per value.  Result valid in thread 0; thread 0 also re-arms the
// ticket.
template <int BS, int NV>
__device__ __forceinline__ void sum_partials(const double *part, int stride, int n, double (&out)[NV],
                                             unsigned int *ticket) {
    __shared__ double sh[NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = warp; k < NV; k += BS / 32) {
        double acc = strided_sum(part + k * stride, lane, n, 32);
        acc = warp_sum(acc);
        if (lane == 0) sh[k] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) out[k] = sh[k];
        *ticket = 0u;
    }
}

}  // namespace hqn
