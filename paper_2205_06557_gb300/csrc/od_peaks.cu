// Pipe micro-benchmarks: the FP32 FMA, MUFU (rsqrt, ex2) and FP64 FMA throughput of this
// GPU, and the latency of a dependent FP64 chain, measured with independent dependency
// chains per thread over a full grid.  These give the ALU roofline denominators of the
// pair kernel (whose work per pair is FP32 FMA-pipe and MUFU instructions) and explain
// the cost of the FP64 sampling code.
#include <cuda_runtime.h>

#include <cmath>

#include "od_internal.h"

namespace od {
namespace peaks {

constexpr int CHAINS = 8;

__global__ void k_ffma(float* out, int iters, float a, float b)
{
    float x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x * 1e-7f + c;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) x[c] = fmaf(x[c], a, b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    if (s == 12345.678f) out[0] = s;
}

// one MUFU function per chain step: rsqrt (0), ex2 of the negated value (1, the negation is
// an operand modifier), rcp (2) and lg2 (3) of the value plus a constant (one FADD)
__global__ void k_mufu(float* out, int iters, int which)
{
    float x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = 0.5f + threadIdx.x * 1e-7f + c * 1e-3f;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) {
            float r;
            if (which == 0)
                asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x[c]));  // converges to 1
            else if (which == 1)
                asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-x[c]));  // stays in (0.5, 1)
            else if (which == 2)
                asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x[c] + 1.0f));  // stays in (0.5, 1)
            else
                asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x[c] + 2.0f));  // stays in (1, 2)
            x[c] = r;
        }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    if (s == 12345.678f) out[0] = s;
}

__global__ void k_dfma(double* out, int iters, double a, double b)
{
    double x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = threadIdx.x * 1e-7 + c;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    if (s == 12345.678) out[0] = s;
}

// one thread, one dependent chain: latency of FP64 fma (which 0) or FP64 exp (which 1)
__global__ void k_dlat(double* out, int iters, int which)
{
    double x = 0.5 + threadIdx.x * 1e-9;
    for (int i = 0; i < iters; ++i) x = which == 0 ? fma(x, 0.999999, 1e-7) : exp(-x) + 0.3;
    out[threadIdx.x] = x;
}

}  // namespace peaks
}  // namespace od

using namespace od::peaks;

extern "C" int od_measure_peaks(double* out)
{
    // out: [0] FFMA  [1] rsqrt  [2] ex2  [3] DFMA  (operations per second per SM)
    //      [4] dependent DFMA latency (ns)  [5] dependent FP64 exp latency (ns)
    //      [6] the device's maximum SM clock (MHz)  [7] rcp  [8] lg2 (operations per second per SM)
    if (!out) return OD_EINVAL;
    int dev = 0, sms = 0, clk_khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return OD_ENODEV;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
    float* fbuf = nullptr;
    double* dbuf = nullptr;
    if (cudaMalloc(&fbuf, 64) != cudaSuccess || cudaMalloc(&dbuf, 1024 * sizeof(double)) != cudaSuccess) return OD_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // 8 CTAs of 256 per SM: 64 warps with 8 independent chains each keep every pipe full
    const int blocks = sms * 8, threads = 256;
    auto time_ms = [&](auto launch) {
        launch();
        cudaEventRecord(e0);
        launch();
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return (double)ms;
    };
    const int it = 4096, it_f = 4 * it;
    const double per_sm = (double)blocks * threads * CHAINS / sms;
    const double t_ffma = time_ms([&] { k_ffma<<<blocks, threads>>>(fbuf, it_f, 1.0000001f, 1e-7f); });
    double t_mufu[4];
    for (int w = 0; w < 4; ++w) t_mufu[w] = time_ms([&] { k_mufu<<<blocks, threads>>>(fbuf, it, w); });
    const double t_dfma = time_ms([&] { k_dfma<<<blocks, threads>>>(dbuf, it / 16, 0.9999999, 1e-7); });
    const int lit = 20000;
    const double t_dlat = time_ms([&] { k_dlat<<<1, 1>>>(dbuf, lit, 0); });
    const double t_dexp = time_ms([&] { k_dlat<<<1, 1>>>(dbuf, lit / 10, 1); });
    out[0] = per_sm * it_f / (t_ffma * 1e-3);
    out[1] = per_sm * it / (t_mufu[0] * 1e-3);
    out[2] = per_sm * it / (t_mufu[1] * 1e-3);
    out[3] = per_sm * (it / 16) / (t_dfma * 1e-3);
    out[4] = t_dlat * 1e6 / lit;
    out[5] = t_dexp * 1e6 / (lit / 10);
    out[6] = clk_khz * 1e-3;
    out[7] = per_sm * it / (t_mufu[2] * 1e-3);
    out[8] = per_sm * it / (t_mufu[3] * 1e-3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(fbuf);
    cudaFree(dbuf);
    return cudaGetLastError() == cudaSuccess ? OD_OK : OD_ECUDA;
}
