// dg_probe.cu -- FMA throughput of the current GPU's CUDA cores, the
// denominator of the roofline fraction of the arithmetic-bound kernels (the
// double-state stage runs on the FP64 pipe).  Not part of the method.
//
// Every thread runs kChains independent multiply-add chains x <- x a + b
// (|a| < 1, so the values stay bounded), so each warp always has independent
// FMAs to issue and the pipe, not the dependency latency, sets the rate.  The
// grid is a whole number of waves of the device (resident CTAs per SM x SM
// count).  One untimed launch, then one launch timed with CUDA events.
#include <cuda_runtime.h>

#include "dg_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(T *out, T a, T b, int iters)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    // a store the compiler cannot drop (s is never exactly -1)
    if (s == T(-1)) out[blockIdx.x] = s;
}

template <typename T>
cudaError_t measure(int iters, double *flop_per_s, double *ms_out)
{
    int dev = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chain_kernel<T>, kThreads, 0);
    if (e != cudaSuccess) return e;
    const long long blocks = (long long)dg::sm_count() * (per_sm > 0 ? per_sm : 1);
    T *out = nullptr;  // never written for these operands; a valid pointer anyway
    e = cudaMalloc(&out, sizeof(T) * blocks);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const T a = T(0.999999), b = T(1e-6);
    if (e == cudaSuccess) {
        fma_chain_kernel<T><<<(unsigned)blocks, kThreads>>>(out, a, b, iters);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) {
        fma_chain_kernel<T><<<(unsigned)blocks, kThreads>>>(out, a, b, iters);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) {
        const double flops = 2.0 * (double)blocks * kThreads * kChains * (double)iters;
        *flop_per_s = flops / (ms * 1e-3);
        if (ms_out) *ms_out = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return e;
}

}  // namespace

extern "C" dg_status dg_fma_throughput(dg_precision precision, double *flop_per_s, double *ms)
{
    if (!flop_per_s) return DG_ERR_ARG;
    cudaError_t e;
    // about 20 ms per launch on a GB300 at either precision (its FP32 rate is
    // ~58x its FP64 rate)
    if (precision == DG_FP64) e = measure<double>(4096, flop_per_s, ms);
    else if (precision == DG_FP32) e = measure<float>(4096 * 64, flop_per_s, ms);
    else return DG_ERR_ARG;
    if (e == cudaErrorMemoryAllocation) return DG_ERR_OOM;
    return e == cudaSuccess ? DG_OK : DG_ERR_CUDA;
}
