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

__global__ void k_mufu(float* out, int iters, int which)
{
    float x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = 1.0f + threadIdx.x * 1e-7f + c * 1e-3f;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) {
            float r;
            if (which == 0) {
                asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x[c]));
                x[c] = r;  // converges to 1
            } else {
                asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x[c]));
                x[c] = r - 1.5f;  // stays bounded (fixed point near -1)
            }
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
    // out: [0] FFMA/clk/SM  [1] rsqrt/clk/SM  [2] ex2/clk/SM  [3] DFMA/clk/SM
    //      [4] dependent DFMA latency (clk)  [5] dependent FP64 exp latency (clk)  [6] SM clock MHz (events)
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
    // clock-normalised rates use a dependent-FMA chain timing as the clock estimate
    const int it = 4096;
    const double total_threads = (double)blocks * threads;
    const double t_ffma = time_ms([&] { k_ffma<<<blocks, threads>>>(fbuf, it, 1.0000001f, 1e-7f); });
    const double t_rsq = time_ms([&] { k_mufu<<<blocks, threads>>>(fbuf, it, 0); });
    const double t_ex2 = time_ms([&] { k_mufu<<<blocks, threads>>>(fbuf, it, 1); });
    const double t_dfma = time_ms([&] { k_dfma<<<blocks, threads>>>(dbuf, it / 16, 0.9999999, 1e-7); });
    const int lit = 20000;
    const double t_dlat = time_ms([&] { k_dlat<<<1, 1>>>(dbuf, lit, 0); });
    const double t_dexp = time_ms([&] { k_dlat<<<1, 1>>>(dbuf, lit / 10, 1); });
    const double f_hz = clk_khz * 1e3;  // nominal; the caller rescales with the measured clock
    const double ops_f = total_threads * it * CHAINS;
    out[0] = ops_f / (t_ffma * 1e-3) / f_hz / sms;
    out[1] = ops_f / (t_rsq * 1e-3) / f_hz / sms;
    out[2] = ops_f / (t_ex2 * 1e-3) / f_hz / sms;
    out[3] = total_threads * (it / 16) * CHAINS / (t_dfma * 1e-3) / f_hz / sms;
    out[4] = t_dlat * 1e-3 * f_hz / lit;
    out[5] = t_dexp * 1e-3 * f_hz / (lit / 10);
    out[6] = clk_khz * 1e-3;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(fbuf);
    cudaFree(dbuf);
    return cudaGetLastError() == cudaSuccess ? OD_OK : OD_ECUDA;
}
