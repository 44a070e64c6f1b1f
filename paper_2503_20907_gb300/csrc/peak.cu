// FP32 pipe throughput of this device, measured: the denominator of the
// projector's "alu" roofline (its work is FP32 fused multiply-adds; the
// device peak SMs x 128 lanes x 2 flops x clock is the derived figure).
//
// Every thread runs kChains independent FMA chains (enough independent work
// to cover the FMA latency with four warps per scheduler) for `iters` steps,
// either as scalar fma.rn.f32 or as packed fma.rn.f32x2 (two FMAs per
// instruction, as the strip kernels' Horner schemes use them).  Results are
// stored so that nothing is dead code.  The caller times the launch.
#include "common.cuh"

namespace spx {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) ffma_peak_kernel(float *out, int iters, float b, float c)
{
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = __fmaf_rn(x[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) ffma2_peak_kernel(float *out, int iters, float b, float c)
{
    unsigned long long x[kChains], bb, cc;
    asm("mov.b64 %0, {%1, %1};" : "=l"(bb) : "f"(b));
    asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        const float v = (float)(threadIdx.x + k) * 1e-3f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[k]) : "f"(v), "f"(-v));
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[k]) : "l"(bb), "l"(cc));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[k]));
        s += lo + hi;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

int64_t fp32_peak_flops(int packed, int blocks, int iters)
{
    // FMAs per thread and step: kChains (scalar) or 2 kChains (packed)
    return (int64_t)blocks * kPeakThreads * iters * kChains * (packed ? 2 : 1) * 2;
}

cudaError_t launch_fp32_peak(int packed, int blocks, int iters, float *out, cudaStream_t s)
{
    // b slightly below 1 keeps the chains finite for any iteration count
    if (packed) ffma2_peak_kernel<<<blocks, kPeakThreads, 0, s>>>(out, iters, 0.999999f, 1e-6f);
    else ffma_peak_kernel<<<blocks, kPeakThreads, 0, s>>>(out, iters, 0.999999f, 1e-6f);
    return cudaGetLastError();
}

}  // namespace spx
