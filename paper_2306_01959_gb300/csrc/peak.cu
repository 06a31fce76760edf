// ALU throughput microbenchmarks: the measured peaks that the roofline of the
// pair kernels is reported against.  The pair pass is bound by plain FP32
// (mixed form) or FP64 (FP64 form) arithmetic, not by HBM or tensor cores, so
// its denominator is the rate of fused multiply-adds this GPU sustains, counted
// as 2 flop each, measured rather than derived from unit counts and clocks.
//
// Each thread runs 8 independent FMA chains (FP32: also as 4 packed FP32x2
// chains, one instruction advancing two); the grid holds 8 CTAs of 256 threads
// per SM.  The result is written only if it equals a value it never takes, so
// nothing is stored and the compiler cannot drop the chains.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "sph.h"

namespace {

__device__ float g_peak_sink_f;
__device__ double g_peak_sink_d;

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_peak_f32(int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        x[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int c = 0; c < kChains; ++c)
                x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += x[c];
    if (s == -1.2345e-30f)
        g_peak_sink_f = s;
}

__global__ void __launch_bounds__(256) k_peak_f32x2(int iters, float a, float b)
{
    float2 x[kChains / 2];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c)
        x[c] = make_float2((float)(threadIdx.x + c), (float)(threadIdx.x + c + 4));
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int c = 0; c < kChains / 2; ++c)
                x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c)
        s += x[c].x + x[c].y;
    if (s == -1.2345e-30f)
        g_peak_sink_f = s;
}

__global__ void __launch_bounds__(256) k_peak_f64(int iters, double a, double b)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        x[c] = (double)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int c = 0; c < kChains; ++c)
                x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += x[c];
    if (s == -1.2345e-300)
        g_peak_sink_d = s;
}

}  // namespace

extern "C" int sph_alu_peak(int32_t precision, int32_t millis, uintptr_t cuda_stream, double *flops_per_s)
{
    if (!flops_per_s || (precision != SPH_FP64 && precision != SPH_MIXED) || millis < 1 || millis > 60000)
        return SPH_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SPH_ECUDA;
    const int blocks = sms * 8, threads = 256;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return SPH_ECUDA;
    // a multiplier below 1 keeps the chains finite for any number of iterations
    const float af = 0.999999f, bf = 1e-3f;
    double best = 0.0;
    const int nkern = precision == SPH_FP64 ? 1 : 2;
    int rc = SPH_OK;
    for (int kern = 0; kern < nkern && rc == SPH_OK; ++kern) {
        auto launch = [&](int iters) {
            if (precision == SPH_FP64)
                k_peak_f64<<<blocks, threads, 0, st>>>(iters, 0.999999999, 1e-6);
            else if (kern == 0)
                k_peak_f32<<<blocks, threads, 0, st>>>(iters, af, bf);
            else
                k_peak_f32x2<<<blocks, threads, 0, st>>>(iters, af, bf);
        };
        // calibrate the iteration count to about `millis` per launch, then time
        // three launches and keep the fastest
        int iters = 64;
        float ms = 0.f;
        for (int tries = 0; tries < 20; ++tries) {
            cudaEventRecord(e0, st);
            launch(iters);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = SPH_ECUDA;
                break;
            }
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms >= 0.5f * millis || iters >= (1 << 26))
                break;
            iters = (int)std::min<double>((double)iters * std::max(2.0, 0.8 * millis / std::max(ms, 1e-3f)),
                                          (double)(1 << 26));
        }
        for (int rep = 0; rep < 3 && rc == SPH_OK; ++rep) {
            cudaEventRecord(e0, st);
            launch(iters);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = SPH_ECUDA;
                break;
            }
            cudaEventElapsedTime(&ms, e0, e1);
            const double flops = 2.0 * kChains * 16.0 * (double)iters * blocks * threads;
            best = std::max(best, flops / (ms * 1e-3));
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == SPH_OK && cudaGetLastError() != cudaSuccess)
        rc = SPH_ECUDA;
    *flops_per_s = best;
    return rc;
}
