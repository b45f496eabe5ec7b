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
#include "dg_kernels.cuh"

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(T *out, T a, T b, int iters)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
#pragma unroll 4
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

// FP64 tensor-core rate: each warp runs kMmaChains independent accumulators
// through mma.sync m8n8k4 (D = A B + C, 8x4 by 4x8 doubles, 512 flop per
// warp instruction).  With `mix`, the odd warps run the FMA chains of
// fma_chain_kernel instead, to see whether the two share one pipe.
constexpr int kMmaChains = 8;

__device__ __forceinline__ void dmma_m8n8k4(double a, double b, double &d0, double &d1)
{
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                 : "+d"(d0), "+d"(d1)
                 : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(kThreads) dmma_kernel(double *out, double a, int iters, int mix,
                                                        double fa, double fb)
{
    const int warp = threadIdx.x >> 5;
    double s = 0.0;
    if (mix && (warp & 1)) {
        double x[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = double(threadIdx.x + c) * 1e-3;
        // the same number of flops per warp as the MMA branch
        const int fit = iters * kMmaChains * 512 / (32 * 2 * kChains);
#pragma unroll 4
        for (int it = 0; it < fit; ++it) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], fa, fb);
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c) s += x[c];
    } else {
        double d0[kMmaChains], d1[kMmaChains];
#pragma unroll
        for (int c = 0; c < kMmaChains; ++c) { d0[c] = 1e-3 * c; d1[c] = 2e-3 * c; }
        const double b = a * 0.5;
#pragma unroll 2
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int c = 0; c < kMmaChains; ++c) dmma_m8n8k4(a, b, d0[c], d1[c]);
        }
#pragma unroll
        for (int c = 0; c < kMmaChains; ++c) s += d0[c] + d1[c];
    }
    if (s == -1.0) out[blockIdx.x] = s;
}

cudaError_t measure_dmma(int iters, int mix, double *flop_per_s, double *ms_out)
{
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dmma_kernel, kThreads, 0);
    if (e != cudaSuccess) return e;
    const long long blocks = (long long)dg::sm_count() * (per_sm > 0 ? per_sm : 1);
    double *out = nullptr;
    e = cudaMalloc(&out, sizeof(double) * blocks);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const double a = 1e-6;  // the accumulators grow by a tiny amount per MMA
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        if (rep == 1) e = cudaEventRecord(e0, 0);
        if (e == cudaSuccess) {
            dmma_kernel<<<(unsigned)blocks, kThreads>>>(out, a, iters, mix, 0.999999, 1e-6);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) {
        // every warp does iters x kMmaChains x 512 flop (mixed: half of them as FMAs)
        const double flops = (double)blocks * (kThreads / 32) * (double)iters * kMmaChains * 512.0;
        *flop_per_s = flops / (ms * 1e-3);
        if (ms_out) *ms_out = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return e;
}

}  // namespace

namespace {
__global__ void __launch_bounds__(256) sqrt_check_kernel(const double *__restrict__ a, double *fast,
                                                         double *ieee, long long n)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    fast[t] = dg::sqrt_pos(a[t]);
    ieee[t] = __dsqrt_rn(a[t]);
}
}  // namespace

extern "C" dg_status dg_selfcheck_sqrt(const double *a, double *fast, double *ieee, int64_t n,
                                       void *stream)
{
    if (!a || !fast || !ieee || n < 0) return DG_ERR_ARG;
    if (n == 0) return DG_OK;
    const long long blocks = (n + 255) / 256;
    if (blocks > 2147483647LL) return DG_ERR_ARG;
    sqrt_check_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(a, fast, ieee,
                                                                                      (long long)n);
    return cudaGetLastError() == cudaSuccess ? DG_OK : DG_ERR_CUDA;
}

extern "C" dg_status dg_dmma_throughput(int mix, double *flop_per_s, double *ms)
{
    if (!flop_per_s || mix < 0 || mix > 1) return DG_ERR_ARG;
    cudaError_t e = measure_dmma(256, mix, flop_per_s, ms);
    if (e == cudaErrorMemoryAllocation) return DG_ERR_OOM;
    return e == cudaSuccess ? DG_OK : DG_ERR_CUDA;
}

extern "C" dg_status dg_fma_throughput(dg_precision precision, double *flop_per_s, double *ms)
{
    if (!flop_per_s) return DG_ERR_ARG;
    cudaError_t e;
    // about 20 ms per launch on a GB300 at either precision (its FP32 rate is
    // ~58x its FP64 rate)
    if (precision == DG_FP64) e = measure<double>(2048, flop_per_s, ms);
    else if (precision == DG_FP32) e = measure<float>(2048 * 64, flop_per_s, ms);
    else return DG_ERR_ARG;
    if (e == cudaErrorMemoryAllocation) return DG_ERR_OOM;
    return e == cudaSuccess ? DG_OK : DG_ERR_CUDA;
}
