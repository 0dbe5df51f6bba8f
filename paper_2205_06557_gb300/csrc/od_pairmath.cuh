// Arithmetic the pair kernels are made of (included by od_device.cuh before the pair
// kernels of od_pairs.cuh): the MUFU approximations and the fixed-point sums of the
// symmetric kernels.  The benchmark ties its recorded DRAM traffic of a pair kernel to a
// hash of this file, od_pairs.cuh and od_internal.h.
#pragma once

#include "od_internal.h"

namespace od {

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ------------------------------------------------ fixed-point pair sums
// A symmetric unit adds its FP32 partial sum v of ion q as round(v 2^K) to a 64-bit
// integer (red.global.add): integer addition is associative, so the total does not depend
// on which CTA evaluates which unit or in what order.  |v 2^K| must stay below 2^60
// (K is set per run from the expected term sum, ~2^30 below it); otherwise ERR_RANGE.
__device__ __forceinline__ void fixed_add(long long* a, float v, float qscale, int* err)
{
    float t = v * qscale;
    if (!(fabsf(t) < 1.152921504606847e18f)) {
        atomicOr(err, t != t ? ERR_NAN : ERR_RANGE);
        t = 0.f;
    }
    atomicAdd((unsigned long long*)a, (unsigned long long)__float2ll_rn(t));
}

__device__ __forceinline__ void fixed_add3(long long* acc, long long ld, long long q, float vx, float vy, float vz,
                                           float qscale, int* err)
{
    fixed_add(acc + q, vx, qscale, err);
    fixed_add(acc + ld + q, vy, qscale, err);
    fixed_add(acc + 2 * ld + q, vz, qscale, err);
}

}  // namespace od
