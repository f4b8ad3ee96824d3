// FP32 and FP64 throughput probes: the denominators of the integrator's
// roofline (FP32) and of the FP64 reductions.
//
// The chain integrator is bound by the FP32 FMA pipe, not by memory or the
// tensor cores, so its peak is the rate at which the SMs retire FP32 fused
// multiply-adds.  Every thread runs eight independent FMA chains
// acc <- acc * a + b (scalar FFMA, or packed f32x2 FFMA2 as the integrator's
// nonbonded loop uses); with full occupancy the chains hide the pipe latency,
// so the time measures issue and pipe throughput alone.  Flops count an FMA
// as two.
#include "internal.h"

namespace pmf {

namespace {

constexpr int kPeakThreads = 512;
constexpr int kPeakChains = 8;

template <bool PACKED> __global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(float *out, int iters, float a, float b)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    float s = 0.f;
    if constexpr (PACKED) {
        const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
        float2 acc[kPeakChains];
#pragma unroll
        for (int k = 0; k < kPeakChains; ++k) acc[k] = make_float2(1e-3f * k, 1e-3f * k + 1e-9f * threadIdx.x);
#pragma unroll 4
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kPeakChains; ++k) acc[k] = __ffma2_rn(acc[k], a2, b2);
        }
#pragma unroll
        for (int k = 0; k < kPeakChains; ++k) s += acc[k].x + acc[k].y;
    } else {
        float acc[kPeakChains];
#pragma unroll
        for (int k = 0; k < kPeakChains; ++k) acc[k] = 1e-3f * k + 1e-9f * threadIdx.x;
#pragma unroll 8
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kPeakChains; ++k) acc[k] = fmaf(acc[k], a, b);
        }
#pragma unroll
        for (int k = 0; k < kPeakChains; ++k) s += acc[k];
    }
    out[tid] = s;  // keeps the chains live
}

// FP64: the same eight chains per thread with DFMA.
__global__ void __launch_bounds__(kPeakThreads) dfma_peak_kernel(double *out, int iters, double a, double b)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    double acc[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) acc[k] = 1e-3 * k + 1e-9 * threadIdx.x;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kPeakChains; ++k) acc[k] = fma(acc[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) s += acc[k];
    out[tid] = s;
}

}  // namespace

cudaError_t fp64_peak_launch(int ctas, int iters, double *out, double *flops, cudaStream_t st)
{
    if (ctas < 1 || iters < 1) return cudaErrorInvalidValue;
    dfma_peak_kernel<<<ctas, kPeakThreads, 0, st>>>(out, iters, 0.999999, 1e-7);
    *flops = (double)ctas * kPeakThreads * (double)iters * kPeakChains * 2.0;
    return cudaGetLastError();
}

// Launches `ctas` CTAs of kPeakThreads threads; out holds ctas x kPeakThreads
// floats.  Returns the flops one launch performs in *flops.
cudaError_t fp32_peak_launch(bool packed, int ctas, int iters, float *out, double *flops, cudaStream_t st)
{
    if (ctas < 1 || iters < 1) return cudaErrorInvalidValue;
    // a < 1 and b small keep every chain bounded (fixed point b / (1 - a))
    const float a = 0.999999f, b = 1e-7f;
    if (packed) fma_peak_kernel<true><<<ctas, kPeakThreads, 0, st>>>(out, iters, a, b);
    else fma_peak_kernel<false><<<ctas, kPeakThreads, 0, st>>>(out, iters, a, b);
    *flops = (double)ctas * kPeakThreads * (double)iters * kPeakChains * (packed ? 4.0 : 2.0);
    return cudaGetLastError();
}

int fp32_peak_threads() { return kPeakThreads; }

}  // namespace pmf
