// mrs_device.cuh -- small device helpers shared by the float32 pair-sum kernels.
#pragma once

#include <cuda_runtime.h>

namespace mrs {

// Approximate reciprocal square root and reciprocal on the SFU (flush-to-zero; the arguments
// here are r^2 + eps^2 > 0).
__device__ __forceinline__ float sfu_rsqrt(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sfu_rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// Kahan step: (sum, comp) += v, with sum - comp the compensated total.
__device__ __forceinline__ void kahan_add(float& sum, float& comp, float v)
{
    const float y = __fsub_rn(v, comp);
    const float t = __fadd_rn(sum, y);
    comp = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
}

// First work unit of CTA p when W units are split into P contiguous ranges.
__device__ __forceinline__ long long unit_start(long long W, int P, int p)
{
    return (W * (long long)p) / (long long)P;
}

}  // namespace mrs
