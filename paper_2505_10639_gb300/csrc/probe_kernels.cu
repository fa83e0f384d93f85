// Throughput probe of the FP32 and FP64 fused multiply-add pipes (see
// include/mfbd_testing.h). Every thread runs 8 independent chains
// x = x * b + c for `iters` iterations; the chains are independent so the
// pipe, not the FMA latency, bounds the rate. The grid fills every SM with
// 8 CTAs of 256 threads (64 warps per SM). The paper has no counterpart: the
// figure is the denominator of the roofline of the FP32-bound kernels and
// of the FP64 part of the frame reduction.
#include <cuda_runtime.h>

#include "../../include/mfbd.h"
#include "../../include/mfbd_testing.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__device__ float g_sink_f;
__device__ double g_sink_d;

__device__ __forceinline__ void sink(float v) { g_sink_f = v; }
__device__ __forceinline__ void sink(double v) { g_sink_d = v; }

template <class T>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(long long iters, T b, T c) {
    T x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = (T)(threadIdx.x + i);
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = x[i] * b + c;
        }
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    // with b, c > 0 every chain stays positive and bounded, so the store
    // never happens; the condition keeps the work alive
    if (s < (T)0) sink(s);
}

template <class T>
int run_probe(int sms, long long iters, void* stream, double* flops, float* ms) {
    const int ctas = 8 * sms;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return MFBD_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return MFBD_ERR_CUDA;
    }
    // warm-up launch, then the timed one
    fma_probe_kernel<T><<<ctas, kThreads, 0, s>>>(iters / 8 + 1, (T)0.5, (T)0.5);
    cudaEventRecord(e0, s);
    fma_probe_kernel<T><<<ctas, kThreads, 0, s>>>(iters, (T)0.5, (T)0.5);
    cudaEventRecord(e1, s);
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float t = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return MFBD_ERR_CUDA;
    *ms = t;
    *flops = 2.0 * kChains * 16.0 * (double)iters * (double)ctas * kThreads;
    return MFBD_OK;
}

}  // namespace

extern "C" int mfbd_probe_fma_rate(int fp64, long long iters, void* stream, double* flops, float* ms) {
    if (!flops || !ms || iters < 1) return MFBD_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MFBD_ERR_UNSUPPORTED;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MFBD_ERR_CUDA;
    return fp64 ? run_probe<double>(sms, iters, stream, flops, ms) : run_probe<float>(sms, iters, stream, flops, ms);
}
