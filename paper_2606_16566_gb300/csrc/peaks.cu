// peaks.cu -- throughput probes of the SM pipes the render is bound by: FP32
// fused multiply-add (scalar FFMA and packed fma.rn.f32x2) and the SFU's
// ex2.approx. They give the measured denominators of the render's roofline
// (work per second against what the GPU sustains at the clock it runs at).
// A measurement utility; the paper has no counterpart.
#include "common.cuh"
#include "host.h"

namespace lgs {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;   // independent dependency chains per thread (hides latency)

// Scalar FMA chains: x = x * m + a, 8 chains per thread; `iters` rounds.
__global__ void __launch_bounds__(PROBE_THREADS) probe_ffma(int iters, float m, float a, float* sink) {
    float x[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = __fmaf_rn(x[k], m, a);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k];
    if (s == 1234.5f) sink[blockIdx.x] = s;   // keeps the chains live; never true in practice
}

// Packed FMA chains (two FP32 FMAs per instruction per lane).
__global__ void __launch_bounds__(PROBE_THREADS) probe_ffma2(int iters, float m, float a, float* sink) {
    float2 x[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k)
        x[k] = make_float2((float)(threadIdx.x + k) * 1e-3f, (float)(threadIdx.x - k) * 1e-3f);
    const float2 m2 = make_float2(m, m), a2 = make_float2(a, a);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = __ffma2_rn(x[k], m2, a2);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k].x + x[k].y;
    if (s == 1234.5f) sink[blockIdx.x] = s;
}

__device__ __forceinline__ float probe_ex2(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ex2 chains: x = 2^(-x) stays in [0.5, 1] for x in [0, 1].
__global__ void __launch_bounds__(PROBE_THREADS) probe_ex2_kernel(int iters, float* sink) {
    float x[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = (float)((threadIdx.x + k) & 63) * (1.f / 64.f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = probe_ex2(-x[k]);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k];
    if (s == 1234.5f) sink[blockIdx.x] = s;
}

}  // namespace lgs

using namespace lgs;

extern "C" lgs_status lgs_peak_probe(int32_t kind, int32_t blocks, int32_t iters, float* d_sink,
                                     double* ops, void* stream) {
    if (!d_sink || !ops || blocks <= 0 || iters <= 0) return LGS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double lanes = (double)blocks * PROBE_THREADS * PROBE_CHAINS * 16.0 * (double)iters;
    switch (kind) {
        case LGS_PROBE_FFMA:
            probe_ffma<<<blocks, PROBE_THREADS, 0, s>>>(iters, 0.999f, 1e-3f, d_sink);
            *ops = 2.0 * lanes;
            break;
        case LGS_PROBE_FFMA2:
            probe_ffma2<<<blocks, PROBE_THREADS, 0, s>>>(iters, 0.999f, 1e-3f, d_sink);
            *ops = 4.0 * lanes;
            break;
        case LGS_PROBE_EX2:
            probe_ex2_kernel<<<blocks, PROBE_THREADS, 0, s>>>(iters, d_sink);
            *ops = lanes;
            break;
        default:
            return LGS_ERR_UNSUPPORTED;
    }
    return cuda_status(cudaGetLastError());
}
