// probe.cu -- throughput of the FP32 FMA pipe and of the FP64 pipe (a measurement aid, not part
// of the method).
//
// The pair-sum kernels are bound by FP32 arithmetic on the CUDA cores; their roofline is the
// FP32 peak 2 x 128 lanes x SMs x clock.  This kernel measures what the FMA pipe sustains on
// the device for three instruction streams: scalar FFMA, packed FFMA2 (fma.rn.f32x2, two lanes
// per instruction, the form the pair-sum kernels use) and the two interleaved one to one; and
// what the float64 pipe sustains for DFMA (the rod kernels are bound by it), with every lane of a
// warp active or only lane 0: the second tells whether the pipe's cost per warp instruction
// depends on the active mask (on GB300 it does not: one lane costs what 32 do).
// Every thread runs 8 independent dependency chains (enough to cover the pipe latency at 8
// warps per scheduler), so the count is issue- and pipe-bound, not latency-bound.
#include "mrs_internal.h"

namespace mrs {
namespace {

constexpr int kProbeBlock = 256;
constexpr int kProbeChains = 8;

// a scalar FMA the compiler cannot pair into a packed one
__device__ __forceinline__ float fma_scalar(float x, float a, float b)
{
    float y;
    asm("fma.rn.f32 %0, %1, %2, %3;" : "=f"(y) : "f"(x), "f"(a), "f"(b));
    return y;
}

// float64: 8 independent DFMA chains per thread, on the first `lanes` lanes of every warp
__global__ void __launch_bounds__(kProbeBlock) dfma_probe_kernel(float* out, int iters, int lanes, double a,
                                                                 double b)
{
    if ((int)(threadIdx.x & 31) >= lanes) return;
    double x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = threadIdx.x * 1e-9 + blockIdx.x * 1e-7 + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

template <int KIND>
__global__ void __launch_bounds__(kProbeBlock) fma_probe_kernel(float* out, int iters, float a, float b)
{
    float2 x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c)
        x[c] = make_float2(threadIdx.x * 1e-7f + c, blockIdx.x * 1e-7f - c);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) {
            if (KIND == 0) {          // scalar: two FFMA per chain and step
                x[c].x = fma_scalar(x[c].x, a, b);
                x[c].y = fma_scalar(x[c].y, a, b);
            } else if (KIND == 1) {   // packed: one FFMA2 per chain and step
                x[c] = __ffma2_rn(x[c], a2, b2);
            } else {                  // alternating scalar pair and packed by chain
                if (c & 1) {
                    x[c] = __ffma2_rn(x[c], a2, b2);
                } else {
                    x[c].x = fma_scalar(x[c].x, a, b);
                    x[c].y = fma_scalar(x[c].y, a, b);
                }
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c].x + x[c].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace mrs

using namespace mrs;

extern "C" int mrs_fma_probe(int device, int kind, int iters, int warps_per_scheduler,
                             double* tflops, float* ms)
{
    clear_error();
    MRS_REQUIRE(kind >= 0 && kind <= 4,
                "kind must be 0 (FFMA), 1 (FFMA2), 2 (mixed), 3 (DFMA) or 4 (DFMA on one lane per warp)");
    MRS_REQUIRE(iters >= 1 && iters <= (1 << 24), "iters must be in 1..2^24");
    MRS_REQUIRE(warps_per_scheduler >= 0 && warps_per_scheduler <= 16,
                "warps_per_scheduler must be in 0..16");
    MRS_REQUIRE(tflops != nullptr, "tflops is NULL");
    MRS_CHECK_CUDA(cudaSetDevice(device));
    int sms = 0, per_sm = 0;
    MRS_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    MRS_CHECK_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, device));
    // 0: every thread slot of every SM (CTAs of kProbeBlock); w >= 1: w CTAs of 128 threads per
    // SM, i.e. w warps on each of the SM's four schedulers
    const int threads = warps_per_scheduler ? 128 : kProbeBlock;
    const int blocks = warps_per_scheduler ? sms * warps_per_scheduler : sms * (per_sm / kProbeBlock);
    float* out = nullptr;
    if (cudaMalloc((void**)&out, sizeof(float) * (size_t)blocks * threads) != cudaSuccess) {
        set_error("probe buffer allocation failed");
        return MRS_ENOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (!e) e = cudaEventCreate(&e1);
    auto launch = [&](int it) {
        if (kind == 0) fma_probe_kernel<0><<<blocks, threads>>>(out, it, 0.999f, 1e-3f);
        else if (kind == 1) fma_probe_kernel<1><<<blocks, threads>>>(out, it, 0.999f, 1e-3f);
        else if (kind == 2) fma_probe_kernel<2><<<blocks, threads>>>(out, it, 0.999f, 1e-3f);
        else dfma_probe_kernel<<<blocks, threads>>>(out, it, kind == 3 ? 32 : 1, 0.999, 1e-3);
        return cudaGetLastError();
    };
    if (!e) e = launch(iters / 8 + 1);   // warm-up
    float t = 0.f;
    if (!e) e = cudaEventRecord(e0);
    if (!e) e = launch(iters);
    if (!e) e = cudaEventRecord(e1);
    if (!e) e = cudaEventSynchronize(e1);
    if (!e) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) {
        set_error("probe failed: %s", cudaGetErrorString(e));
        return MRS_ECUDA;
    }
    // every chain step is two FP32 lane FMAs (two flops each) in kinds 0..2, one DFMA in kind 3
    // and kind 4; kind 4 counts the active lanes only (one per warp)
    const double lanes = kind == 4 ? (double)blocks * (threads / 32) : (double)blocks * threads;
    const double flops = (kind >= 3 ? 2.0 : 4.0) * kProbeChains * (double)iters * lanes;
    *tflops = flops / (t * 1e-3) / 1e12;
    if (ms) *ms = t;
    return MRS_OK;
}
