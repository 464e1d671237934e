// Throughput microbenchmarks of the arithmetic units the hot path leans on:
// FP32 FMA, FP64 FMA, and the multi-function unit (rsqrt, sin).  They give the
// measured denominators of the ALU rooflines.  Measurement utility only.
#include <cuda_runtime.h>

#include "../../include/rlf_peaks.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void fma32_kernel(float *out, int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3f + c;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    float s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void fma32x2_kernel(float *out, int iters, float a, float b)
{
    unsigned long long x[kChains];
    unsigned long long av, bv;
    asm("mov.b64 %0, {%1, %2};" : "=l"(av) : "f"(a), "f"(a));
    asm("mov.b64 %0, {%1, %2};" : "=l"(bv) : "f"(b), "f"(b));
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        const float x0 = threadIdx.x * 1e-3f + c, x1 = x0 + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(x0), "f"(x1));
    }
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(av), "l"(bv));
    float s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        float x0, x1;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(x0), "=f"(x1) : "l"(x[c]));
        s += x0 + x1;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void fma64_kernel(double *out, int iters, double a, double b)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3 + c;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    double s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void rsqrt_kernel(float *out, int iters)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.5f + threadIdx.x * 1e-3f + c;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = rsqrtf(x[c]);
    float s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void sin_kernel(float *out, int iters)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 0.3f + threadIdx.x * 1e-4f + c * 0.1f;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = __sinf(x[c]);
    float s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename F>
double time_ms(F launch, cudaStream_t st)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    launch();  // warm-up
    cudaEventRecord(a, st);
    launch();
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

}  // namespace

extern "C" int rlf_peaks_measure(void *scratch, size_t scratch_bytes, void *stream, rlf_peaks *out)
{
    if (!scratch || !out) return 1;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8;
    const size_t need = (size_t)blocks * kThreads * sizeof(double);
    if (scratch_bytes < need) return 2;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float *f = static_cast<float *>(scratch);
    double *d = static_cast<double *>(scratch);
    const double threads = (double)blocks * kThreads;
    const int it32 = 4096, it64 = 128, itmu = 1024;
    double ms;
    ms = time_ms([&] { fma32_kernel<<<blocks, kThreads, 0, st>>>(f, it32, 0.999999f, 1e-7f); }, st);
    out->fp32_fma_per_s = threads * it32 * kChains / (ms * 1e-3);
    ms = time_ms([&] { fma32x2_kernel<<<blocks, kThreads, 0, st>>>(f, it32, 0.999999f, 1e-7f); }, st);
    out->fp32x2_fma_per_s = 2.0 * threads * it32 * kChains / (ms * 1e-3);
    ms = time_ms([&] { fma64_kernel<<<blocks, kThreads, 0, st>>>(d, it64, 0.999999, 1e-7); }, st);
    out->fp64_fma_per_s = threads * it64 * kChains / (ms * 1e-3);
    ms = time_ms([&] { rsqrt_kernel<<<blocks, kThreads, 0, st>>>(f, itmu); }, st);
    out->mufu_rsqrt_per_s = threads * itmu * kChains / (ms * 1e-3);
    ms = time_ms([&] { sin_kernel<<<blocks, kThreads, 0, st>>>(f, itmu); }, st);
    out->mufu_sin_per_s = threads * itmu * kChains / (ms * 1e-3);
    out->sm_count = sms;
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}
