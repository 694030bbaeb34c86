// hqn_measure_peak: the device's non-tensor FMA throughput, measured.  The
// roofline of the tet pass (and of any FLOP-bound stage) needs the CUDA
// cores' peak; nominal figures assume the maximum clock, while a loaded part
// may run below it, so the peak is measured on the device itself.
//
// Every thread runs kChains independent chains x <- x * a + b of fused
// multiply-adds (no two of a chain's operations can overlap, but the chains
// of a thread and the warps of an SM can), on enough blocks to fill every SM.
#include <cuda_runtime.h>

#include "../../include/hqn.h"

namespace hqn {
void set_last_error(const char *msg);  // api.cu
}

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

template <typename R>
__global__ void __launch_bounds__(kThreads) k_fma_chains(R *sink, int iters, R a, R b) {
    R x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = R(threadIdx.x + k) * R(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    }
    R s = R(0);
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == R(-1.25)) sink[blockIdx.x] = s;  // keeps the chains live; never true for these inputs
}

template <typename R>
int measure(double *flops_per_s) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HQN_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HQN_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<R>, kThreads, 0) != cudaSuccess)
        return HQN_ERR_CUDA;
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    // |a| < 1 keeps every chain bounded: x converges to b / (1 - a)
    const R a = R(0.999), b = R(1e-4);
    R *sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = HQN_ERR_CUDA;
    float ms = 0.f;
    int iters = 1 << 12;
    if (cudaMalloc(&sink, sizeof(R) * (size_t)blocks) != cudaSuccess) goto out;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) goto out;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) goto out;
    // grow the chains until one launch runs for at least 20 ms
    for (;;) {
        k_fma_chains<R><<<blocks, kThreads, 0, st>>>(sink, iters, a, b);  // warm-up at this length
        cudaEventRecord(e0, st);
        k_fma_chains<R><<<blocks, kThreads, 0, st>>>(sink, iters, a, b);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) goto out;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) goto out;
        if (ms >= 20.f || iters >= (1 << 24)) break;
        iters *= 2;
    }
    if (cudaGetLastError() != cudaSuccess) goto out;
    *flops_per_s = 2.0 * kChains * (double)iters * kThreads * blocks / (ms * 1e-3);
    rc = HQN_OK;
out:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (sink) cudaFree(sink);
    if (rc != HQN_OK) hqn::set_last_error("hqn_measure_peak: a CUDA call failed");
    return rc;
}

}  // namespace

extern "C" int hqn_measure_peak(int32_t precision, double *flops_per_s) {
    if (!flops_per_s || (precision != HQN_FP32_MIXED && precision != HQN_FP64_PLAIN)) {
        hqn::set_last_error("hqn_measure_peak: bad argument");
        return HQN_ERR_ARG;
    }
    return precision == HQN_FP32_MIXED ? measure<float>(flops_per_s) : measure<double>(flops_per_s);
}
