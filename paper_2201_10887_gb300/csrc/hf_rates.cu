// Measured rates of the arithmetic units the discretization and the ray walk
// are designed against (hf_measure_unit_rates): MUFU ex2 and FP32 FMA
// throughput summed over the SMs, and the SM count.  Each thread runs eight
// independent dependency chains so that the unit, not the chain latency,
// sets the pace; one CTA of 256 threads per quarter SM slot keeps 32 warps
// per SM in flight.
#include <cuda_runtime.h>

#include "hf_internal.h"

namespace hfi {
namespace {

constexpr int kRateChains = 8;
constexpr int kRateIters = 4096;
constexpr int kRateCtasPerSm = 4;

__device__ float g_rate_sink[256];  // written only if a chain ends on an impossible value

__device__ __forceinline__ float ex2_ftz(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// x <- 2^-x: the chain settles at the fixed point near 0.641.
__global__ void __launch_bounds__(256) k_rate_ex2(float seed) {
    float x[kRateChains];
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) x[c] = -0.01f * float(c + 1) - seed * float(threadIdx.x & 7);
    for (int it = 0; it < kRateIters; ++it) {
#pragma unroll
        for (int c = 0; c < kRateChains; ++c) x[c] = ex2_ftz(-x[c]);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) s += x[c];
    if (s == 123.456f) g_rate_sink[threadIdx.x] = s;  // keeps the chains live
}

// x <- x * a + b with |a| < 1: settles at b / (1 - a) = 1.
__global__ void __launch_bounds__(256) k_rate_ffma(float seed) {
    float x[kRateChains];
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) x[c] = seed + float(c) * 0.125f + float(threadIdx.x & 7);
    const float a = 0.999f - seed, b = 0.001f;
    for (int it = 0; it < kRateIters; ++it) {
#pragma unroll
        for (int c = 0; c < kRateChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) s += x[c];
    if (s == 123.456f) g_rate_sink[threadIdx.x] = s;
}

// Best of three timed launches after one warm-up, in operations per second.
template <class K>
int time_rate(K kernel, int sms, cudaStream_t s, double* out) {
    const dim3 grid(unsigned(sms * kRateCtasPerSm)), block(256);
    cudaEvent_t a = nullptr, b = nullptr;
    int e = cudaEventCreate(&a);
    if (!e) e = cudaEventCreate(&b);
    float best = 0.f;
    for (int rep = 0; rep < 4 && !e; ++rep) {
        e = cudaEventRecord(a, s);
        if (!e) {
            kernel<<<grid, block, 0, s>>>(0.0f);
            e = cudaGetLastError();
        }
        if (!e) e = cudaEventRecord(b, s);
        if (!e) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (!e) e = cudaEventElapsedTime(&ms, a, b);
        if (!e && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (!e) *out = double(grid.x) * block.x * kRateIters * kRateChains / (double(best) * 1e-3);
    return e;
}

}  // namespace

int measure_unit_rates(double* ex2_per_s, double* ffma_per_s, int* sm_count, void* stream) {
    int dev = 0, sms = 0;
    int e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const cudaStream_t s = cudaStream_t(stream);
    if (!e) e = time_rate(k_rate_ex2, sms, s, ex2_per_s);
    if (!e) e = time_rate(k_rate_ffma, sms, s, ffma_per_s);
    if (!e) *sm_count = sms;
    return e;
}

}  // namespace hfi
