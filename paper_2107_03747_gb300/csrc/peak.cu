// peak.cu -- FMA-pipe microbenchmark: the FP32 / FP64 vector peak that bounds the flow kernels.
//
// Every thread runs 8 independent fused multiply-add chains (enough instruction-level
// parallelism to fill the pipe) for `iters` iterations; 2 flops per FMA.  The grid is
// `blocks_per_sm` x (number of SMs) blocks of 256 threads.  The result is written to a
// caller-owned sink so the chains cannot be removed.  The packed FP32 variant runs the same
// chains on fma.rn.f32x2 pairs (two FMAs per instruction): it checks that the packed form the
// FP32 flow kernels use does not deliver more than the scalar peak, which would make that the
// roofline denominator instead.
#include <cuda_runtime.h>

#include "../../include/tgf.h"

namespace {

template <class T>
__global__ void __launch_bounds__(256) k_fma(T* sink, int iters, T a, T b) {
    T x0 = T(threadIdx.x) * T(1e-7), x1 = x0 + T(1), x2 = x0 + T(2), x3 = x0 + T(3);
    T x4 = x0 + T(4), x5 = x0 + T(5), x6 = x0 + T(6), x7 = x0 + T(7);
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
            x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
        }
    }
    T s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (s == T(-12345.678)) sink[blockIdx.x] = s;
}

// 8 independent chains of packed pairs: 16 FMAs per unrolled row
__global__ void __launch_bounds__(256) k_fma_x2(float* sink, int iters, float a, float b) {
    unsigned long long x[8], av, bv;
    asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float lo = float(threadIdx.x) * 1e-7f + float(2 * k), hi = lo + 1.f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[k]) : "f"(lo), "f"(hi));
    }
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < 8; ++k) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[k]) : "l"(av), "l"(bv));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[k]));
        s += lo + hi;
    }
    if (s == -12345.678f) sink[blockIdx.x] = s;
}

// 8 packed chains and 8 scalar chains interleaved (24 FMAs per unrolled row): whether packed and
// scalar FMAs of one warp scheduler overlap on its two FMA pipes
__global__ void __launch_bounds__(256) k_fma_mixed(float* sink, int iters, float a, float b) {
    unsigned long long x[8], av, bv;
    float y[8];
    asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float lo = float(threadIdx.x) * 1e-7f + float(2 * k), hi = lo + 1.f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[k]) : "f"(lo), "f"(hi));
        y[k] = lo + 0.5f;
    }
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[k]) : "l"(av), "l"(bv));
                y[k] = fmaf(y[k], a, b);
            }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[k]));
        s += lo + hi + y[k];
    }
    if (s == -12345.678f) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" tgf_status tgf_fma_peak(int prec, void* sink_dev, int blocks_per_sm, int iters, double* tflops,
                                   void* stream) {
    if ((prec != TGF_FP64 && prec != TGF_FP32 && prec != TGF_FMA_PEAK_FP32X2 && prec != TGF_FMA_PEAK_FP32_MIXED) ||
        !sink_dev || blocks_per_sm < 1 || iters < 1 || !tflops)
        return TGF_EINVAL;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TGF_ECUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TGF_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = nsm * blocks_per_sm;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return TGF_ECUDA;
    auto launch = [&]() {
        if (prec == TGF_FP64)
            k_fma<double><<<grid, 256, 0, st>>>((double*)sink_dev, iters, 0.999999, 1e-9);
        else if (prec == TGF_FMA_PEAK_FP32X2)
            k_fma_x2<<<grid, 256, 0, st>>>((float*)sink_dev, iters, 0.999999f, 1e-9f);
        else if (prec == TGF_FMA_PEAK_FP32_MIXED)
            k_fma_mixed<<<grid, 256, 0, st>>>((float*)sink_dev, iters, 0.999999f, 1e-9f);
        else
            k_fma<float><<<grid, 256, 0, st>>>((float*)sink_dev, iters, 0.999999f, 1e-9f);
    };
    launch();  // warm-up
    cudaEventRecord(e0, st);
    launch();
    cudaEventRecord(e1, st);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess || ms <= 0.f) return TGF_ECUDA;
    const double fmas_per_row = prec == TGF_FMA_PEAK_FP32X2 ? 16.0 : prec == TGF_FMA_PEAK_FP32_MIXED ? 24.0 : 8.0;
    const double flops = 2.0 * fmas_per_row * 16.0 * (double)iters * 256.0 * (double)grid;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return TGF_OK;
}
