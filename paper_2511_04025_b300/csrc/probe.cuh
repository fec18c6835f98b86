// probe.cuh -- arithmetic peak probes of the device (FP32 FMA, packed FP32x2
// FMA, FP64 FMA).  They give the field kernel (FP64-bound) and the CUDA-core
// stiffness apply a measured arithmetic ceiling beside the measured copy rate
// and GEMM rate.  Each thread runs kChains independent FMA chains (enough to
// cover the pipe latency) for `iters` rounds; the result is folded into one
// store per thread so the compiler keeps every FMA.
#pragma once

#include "common.cuh"

namespace shl {

constexpr int kProbeChains = 8;

__global__ void probe_ffma_kernel(int iters, float a, float b, float *out) {
    float acc[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) acc[c] = (float)(threadIdx.x + c);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) acc[c] = fmaf(acc[c], a, b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += acc[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void probe_ffma2_kernel(int iters, float a, float b, float *out) {
    float2 acc[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) acc[c] = make_float2((float)threadIdx.x, (float)c);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) acc[c] = __ffma2_rn(acc[c], a2, b2);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += acc[c].x + acc[c].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void probe_dfma_kernel(int iters, double a, double b, float *out) {
    double acc[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) acc[c] = (double)(threadIdx.x + c);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) acc[c] = fma(acc[c], a, b);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += acc[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

}  // namespace shl
