// Device code of the pair forces (Eq. 1's ion-ion term), included by od_device.cuh after
// its helpers: the pair coefficient (plain and with the cutoff's switching function), the
// ordered-pair kernel, the symmetric kernels (scalar and on packed FP32 pairs) and the
// units the batched kernel and the cutoff reuse.
#pragma once

namespace od {

// ------------------------------------------------------------ pair forces
// block g of G owns units [g U / G, (g+1) U / G); this is the block owning unit u
__device__ __forceinline__ int owner_of(long long u, long long U, int G)
{
    return (int)(((u + 1) * (long long)G - 1) / U);
}

// Pair coefficient in scaled coordinates s = r log2(e) / lambda_De, which make
// exp(-r/lambda) = 2^-s and 1 + r/lambda = 1 + s ln 2.  For d = s_j - s_i and
// r2 = |d|^2 + eps (eps keeps a self pair finite: its d is exactly 0) the term of Eq. 1's
// ion-ion part is d (1 + s ln2) 2^-s / s^3.  With ri = 1/s, (1 + s ln2) ri^3 =
// ri^2 (ri + ln2) since s ri = 1 (up to the rsqrt rounding, 2e-7 relative), one product
// fewer than the literal form.
__device__ __forceinline__ float pair_c3(float dx, float dy, float dz)
{
    constexpr float EPS2 = 1e-24f;
    constexpr float LN2 = 0.69314718055994531f;
    float r2 = fmaf(dx, dx, EPS2);
    r2 = fmaf(dy, dy, r2);
    r2 = fmaf(dz, dz, r2);
    const float ri = rsqrt_approx(r2);
    const float e = ex2_approx(-(r2 * ri));
    return (e * (ri * ri)) * (ri + LN2);
}

// pair_c3 with the ion-ion cutoff (Sec. 5; the switching form is a reading): the pair
// energy is multiplied by S(x) = 1 - 10 x^3 + 15 x^4 - 6 x^5, x = (s - s0) w_inv clamped to
// [0, 1], and the force is minus the gradient of the switched energy.  In the scaled
// units of pair_c3 this is c3 = e ri^2 [(ri + ln2) S(x) - S'(x) w_inv], with
// S'(x) = -30 x^2 (1 - x)^2.  The clamp makes it exactly the plain term for s <= s0 and
// exactly 0 from the cutoff on (S(1) = S'(1) = 0); there is no branch.
__device__ __forceinline__ float switch_bracket(float s, float ri, float s0, float w_inv)
{
    constexpr float LN2 = 0.69314718055994531f;
    const float x = fminf(fmaxf((s - s0) * w_inv, 0.f), 1.f);
    const float x2 = x * x, y = 1.f - x;
    const float S = fmaf(-(x2 * x), fmaf(fmaf(6.f, x, -15.f), x, 10.f), 1.f);
    const float dS = -30.f * x2 * (y * y);
    return fmaf(ri + LN2, S, -dS * w_inv);
}

__device__ __forceinline__ float pair_c3_cut(float dx, float dy, float dz, float s0, float w_inv)
{
    constexpr float EPS2 = 1e-24f;
    float r2 = fmaf(dx, dx, EPS2);
    r2 = fmaf(dy, dy, r2);
    r2 = fmaf(dz, dz, r2);
    const float ri = rsqrt_approx(r2);
    const float s = r2 * ri;
    const float e = ex2_approx(-s);
    return (e * (ri * ri)) * switch_bracket(s, ri, s0, w_inv);
}

// Accumulate into IPT targets per thread the pair terms of sources [j0, j1), staged
// through shared memory BT at a time (acc += d c3, c3 from pair_c3, or from pair_c3_cut
// with the switching zone s0, w_inv when CUT).
template <int BT, int IPT, bool CUT = false>
__device__ __forceinline__ void pair_chunk(const float4* __restrict__ fpos, int j0, int j1, const float* xi,
                                           const float* yi, const float* zi, float* ax, float* ay, float* az,
                                           float4* sj, float s0 = 0.f, float w_inv = 0.f)
{
    for (int jb = j0; jb < j1; jb += BT) {
        __syncthreads();
        sj[threadIdx.x] = fpos[jb + threadIdx.x];
        __syncthreads();
        // blocked summation: each shared tile of BT sources is summed on its own and
        // then added to the running sum, so the FP32 rounding error grows like
        // sqrt(BT) + sqrt(n / BT) instead of sqrt(n) over n same-sign terms
        float bx[IPT], by[IPT], bz[IPT];
#pragma unroll
        for (int k = 0; k < IPT; ++k) bx[k] = by[k] = bz[k] = 0.f;
#pragma unroll 8
        for (int jj = 0; jj < BT; ++jj) {
            const float4 pj = sj[jj];
#pragma unroll
            for (int k = 0; k < IPT; ++k) {
                const float dx = pj.x - xi[k], dy = pj.y - yi[k], dz = pj.z - zi[k];
                const float c3 = CUT ? pair_c3_cut(dx, dy, dz, s0, w_inv) : pair_c3(dx, dy, dz);
                bx[k] = fmaf(c3, dx, bx[k]);
                by[k] = fmaf(c3, dy, by[k]);
                bz[k] = fmaf(c3, dz, bz[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            ax[k] += bx[k];
            ay[k] += by[k];
            az[k] += bz[k];
        }
    }
}

// Persistent all-pairs kernel: block g of G takes a contiguous range of (target tile,
// source chunk) units, accumulates in registers across the chunks of a tile and writes
// one partial per tile segment (slot = g - owner of the tile's first unit).
template <int BT, int IPT>
__global__ void __launch_bounds__(BT) k_forces(const float4* __restrict__ fpos, float4* __restrict__ part, ForceArgs F)
{
    __shared__ float4 sj[BT];
    const int g = blockIdx.x;
    long long u = (long long)g * F.U / F.G;
    const long long u_end = (long long)(g + 1) * F.U / F.G;
    while (u < u_end) {
        const int t = (int)(u / F.JS);
        const long long u_tile_end = min(u_end, (long long)(t + 1) * F.JS);
        float xi[IPT], yi[IPT], zi[IPT], ax[IPT], ay[IPT], az[IPT];
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const float4 p = fpos[t * F.TI + k * BT + threadIdx.x];
            xi[k] = p.x;
            yi[k] = p.y;
            zi[k] = p.z;
            ax[k] = 0.f;
            ay[k] = 0.f;
            az[k] = 0.f;
        }
        for (; u < u_tile_end; ++u) {
            const int c = (int)(u % F.JS);
            const int j0 = c * F.JC;
            const int j1 = min(j0 + F.JC, F.n_pad);
            pair_chunk<BT, IPT>(fpos, j0, j1, xi, yi, zi, ax, ay, az, sj);
        }
        const int slot = g - owner_of((long long)t * F.JS, F.U, F.G);
        float4* out = part + (long long)slot * F.n_pad + t * F.TI + threadIdx.x;
#pragma unroll
        for (int k = 0; k < IPT; ++k) out[k * BT] = make_float4(ax[k], ay[k], az[k], 0.f);
    }
}

// Unit u of the row-major upper triangle of T x T tiles (J >= I), where row I starts
// at I T - I (I - 1) / 2.
__device__ __forceinline__ void tri_unit(long long u, int T, int& I, int& J)
{
    const double b = 2.0 * T + 1.0;
    long long i = (long long)((b - sqrt(fmax(b * b - 8.0 * (double)u, 0.0))) * 0.5);
    i = max(0ll, min(i, (long long)T - 1));
    while (i > 0 && i * T - i * (i - 1) / 2 > u) --i;
    while (i + 1 < T && (i + 1) * T - (i + 1) * i / 2 <= u) ++i;
    I = (int)i;
    J = (int)(I + (u - (i * T - i * (i - 1) / 2)));
}

// Symmetric (Newton III) all-pairs kernel: each unordered pair is evaluated once and
// applied to both ions.  Tiles of TI = BT IPT ions; units are the tile pairs (I, J >= I)
// in row-major order, split into contiguous ranges over the persistent blocks (the packed
// kernel k_forces_sym2 takes them from a dynamic queue instead).
//
// Unit (I, J > I): warp w holds 32 IPT targets of tile I (IPT per lane) and walks tile J
// in groups of 32 sources, one per lane.  Each source travels round the warp by shuffles
// together with its own accumulator, so after 32 rotations every lane has met every
// source of the group and each accumulator is back on its lane.  The source-side sums of
// the warps are combined in shared memory in a fixed warp order, SUB sources at a time
// (double buffered, one barrier per SUB sources).
// Unit (I, I): the ordered pairs of the tile through pair_chunk (the self pair is 0).
//
// Sums: the unit's FP32 target-side sums (ions of tile I) and source-side sums (ions of
// tile J) are added to the ions' fixed-point accumulators (fixed_add3), so the result
// does not depend on the order in which units finish; the kick reads and clears them.
template <int BT, int IPT>
__global__ void __launch_bounds__(BT) k_forces_sym(const float4* __restrict__ fpos, ForceArgs F)
{
    constexpr int NW = BT / 32;
    constexpr int TI = BT * IPT;
    constexpr int SUB = 128;
    static_assert(TI % SUB == 0 && (TI / SUB) % 2 == 0, "tile must hold an even number of combine steps");
    __shared__ float s_acc[2][3][NW][SUB];
    __shared__ float4 sj[BT];
    const int T = F.JS;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int src = (lane + 1) & 31;
    long long u = (long long)blockIdx.x * F.U / F.G;
    const long long u_end = (long long)(blockIdx.x + 1) * F.U / F.G;
    if (u >= u_end) return;
    int I, J;
    tri_unit(u, T, I, J);
    for (; u < u_end; ++u) {
        float xi[IPT], yi[IPT], zi[IPT], ax[IPT], ay[IPT], az[IPT];
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const float4 p = fpos[I * TI + k * BT + threadIdx.x];
            xi[k] = p.x;
            yi[k] = p.y;
            zi[k] = p.z;
            ax[k] = 0.f;
            ay[k] = 0.f;
            az[k] = 0.f;
        }
        if (I == J) {
            pair_chunk<BT, IPT>(fpos, I * TI, I * TI + TI, xi, yi, zi, ax, ay, az, sj);
        } else {
            const int jb = J * TI;
            for (int sc = 0; sc < TI / SUB; ++sc) {
                const int buf = sc & 1;
#pragma unroll 1
                for (int q = 0; q < SUB / 32; ++q) {
                    const float4 pj = __ldg(fpos + jb + sc * SUB + q * 32 + lane);
                    float xj = pj.x, yj = pj.y, zj = pj.z, bx = 0.f, by = 0.f, bz = 0.f;
#pragma unroll 4
                    for (int r = 0; r < 32; ++r) {
#pragma unroll
                        for (int k = 0; k < IPT; ++k) {
                            const float dx = xj - xi[k], dy = yj - yi[k], dz = zj - zi[k];
                            const float c3 = pair_c3(dx, dy, dz);
                            ax[k] = fmaf(c3, dx, ax[k]);
                            ay[k] = fmaf(c3, dy, ay[k]);
                            az[k] = fmaf(c3, dz, az[k]);
                            bx = fmaf(-c3, dx, bx);
                            by = fmaf(-c3, dy, by);
                            bz = fmaf(-c3, dz, bz);
                        }
                        xj = __shfl_sync(0xffffffffu, xj, src);
                        yj = __shfl_sync(0xffffffffu, yj, src);
                        zj = __shfl_sync(0xffffffffu, zj, src);
                        bx = __shfl_sync(0xffffffffu, bx, src);
                        by = __shfl_sync(0xffffffffu, by, src);
                        bz = __shfl_sync(0xffffffffu, bz, src);
                    }
                    s_acc[buf][0][w][q * 32 + lane] = bx;
                    s_acc[buf][1][w][q * 32 + lane] = by;
                    s_acc[buf][2][w][q * 32 + lane] = bz;
                }
                // the other buffer's readers (previous combine step) finished before they
                // reached this barrier, so the next step may refill it without another one
                __syncthreads();
                for (int j = threadIdx.x; j < SUB; j += BT) {
                    float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
                    for (int ww = 0; ww < NW; ++ww) {
                        sx += s_acc[buf][0][ww][j];
                        sy += s_acc[buf][1][ww][j];
                        sz += s_acc[buf][2][ww][j];
                    }
                    fixed_add3(F.psum, F.psum_ld, jb + sc * SUB + j, sx, sy, sz, F.qscale, F.err);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < IPT; ++k)
            fixed_add3(F.psum, F.psum_ld, I * TI + k * BT + threadIdx.x, ax[k], ay[k], az[k], F.qscale, F.err);
        if (++J == T) J = ++I;
    }
}

// ---------------------------------------- packed FP32 pairs (f32x2, sm_100 family)
// Two FP32 values in one 64-bit register pair; add/sub/mul/fma on both in one
// instruction with the same IEEE round-to-nearest as the scalar forms.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk2(float a, float b)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ void upk2(f32x2 v, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }

__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// pair_c3 for two pairs at once (same operations and rounding per lane of the pair)
__device__ __forceinline__ f32x2 pair_c3x2(f32x2 dx, f32x2 dy, f32x2 dz)
{
    const f32x2 eps2 = pk2(1e-24f, 1e-24f), ln2 = pk2(0.69314718055994531f, 0.69314718055994531f);
    f32x2 r2 = fma2(dx, dx, eps2);
    r2 = fma2(dy, dy, r2);
    r2 = fma2(dz, dz, r2);
    float ra, rb;
    upk2(r2, ra, rb);
    const f32x2 ri = pk2(rsqrt_approx(ra), rsqrt_approx(rb));
    float sa, sb;
    upk2(mul2(r2, ri), sa, sb);
    const f32x2 e = pk2(ex2_approx(-sa), ex2_approx(-sb));
    return mul2(mul2(e, mul2(ri, ri)), add2(ri, ln2));
}

// switch_bracket for two pairs at once, in packed operations (only the clamp is per
// lane): x = (s - s0) w_inv in [0, 1], S = 1 + x^3 (15 x - 6 x^2 - 10),
// -S' = 30 x^2 (1 - x)^2, bracket = (ri + ln2) S + 30 w_inv x^2 (1 - x)^2
__device__ __forceinline__ f32x2 switch_bracket2(f32x2 s, f32x2 ri, float s0, float w_inv)
{
    constexpr float LN2 = 0.69314718055994531f;
    f32x2 x = fma2(s, pk2(w_inv, w_inv), pk2(-s0 * w_inv, -s0 * w_inv));
    float xa, xb;
    upk2(x, xa, xb);
    x = pk2(fminf(fmaxf(xa, 0.f), 1.f), fminf(fmaxf(xb, 0.f), 1.f));
    const f32x2 x2 = mul2(x, x);
    const f32x2 t = fma2(fma2(x, pk2(-6.f, -6.f), pk2(15.f, 15.f)), x, pk2(-10.f, -10.f));
    const f32x2 S = fma2(mul2(x2, x), t, pk2(1.f, 1.f));
    const f32x2 y2 = fma2(x, add2(x, pk2(-2.f, -2.f)), pk2(1.f, 1.f));
    return fma2(mul2(x2, y2), pk2(30.f * w_inv, 30.f * w_inv), mul2(add2(ri, pk2(LN2, LN2)), S));
}

// pair_c3_cut for two pairs at once: the packed plain coefficient's steps, then the
// packed switching bracket
__device__ __forceinline__ f32x2 pair_c3x2_cut(f32x2 dx, f32x2 dy, f32x2 dz, float s0, float w_inv)
{
    const f32x2 eps2 = pk2(1e-24f, 1e-24f);
    f32x2 r2 = fma2(dx, dx, eps2);
    r2 = fma2(dy, dy, r2);
    r2 = fma2(dz, dz, r2);
    float ra, rb;
    upk2(r2, ra, rb);
    const f32x2 ri = pk2(rsqrt_approx(ra), rsqrt_approx(rb));
    const f32x2 s = mul2(r2, ri);
    float sa, sb;
    upk2(s, sa, sb);
    const f32x2 e = pk2(ex2_approx(-sa), ex2_approx(-sb));
    return mul2(mul2(e, mul2(ri, ri)), switch_bracket2(s, ri, s0, w_inv));
}

constexpr int SYM_SUB = 128;  // sources per combine step of the symmetric kernels

// One tile-pair unit (I, J >= I) of the symmetric kernel with packed FP32 pairs: the same
// units, fixed-point sums and fixed combine order as k_forces_sym, but the travelling packet holds
// two sources (the lane's sources q*64 + lane and q*64 + 32 + lane of the group), each
// target is duplicated into both halves of a pair, and every FP32 operation of the pair
// term acts on the two sources in one instruction.  Source-side sums are accumulated
// with the target-side sign and negated when the warps' sums are combined.  Every unit
// starts on combine buffer 0 and ends on buffer 1, so consecutive units need no barrier
// between them beyond the one per combine step.
template <int BT, int IPT, bool CUT = false>
__device__ __forceinline__ void sym2_unit(const float4* __restrict__ fpos, const ForceArgs& F, int I, int J,
                                          float (&s_acc)[2][3][BT / 32][SYM_SUB], float4* sj)
{
    constexpr int NW = BT / 32;
    constexpr int TI = BT * IPT;
    static_assert(TI % SYM_SUB == 0 && (TI / SYM_SUB) % 2 == 0, "tile must hold an even number of combine steps");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int src = (lane + 1) & 31;
    float xi[IPT], yi[IPT], zi[IPT], ax[IPT], ay[IPT], az[IPT];
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
        const float4 p = fpos[I * TI + k * BT + threadIdx.x];
        xi[k] = p.x;
        yi[k] = p.y;
        zi[k] = p.z;
        ax[k] = 0.f;
        ay[k] = 0.f;
        az[k] = 0.f;
    }
    if (I == J) {
        pair_chunk<BT, IPT, CUT>(fpos, I * TI, I * TI + TI, xi, yi, zi, ax, ay, az, sj, F.cut_s0, F.cut_inv_w);
    } else {
        f32x2 xd[IPT], yd[IPT], zd[IPT], ax2[IPT], ay2[IPT], az2[IPT];
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            xd[k] = pk2(xi[k], xi[k]);
            yd[k] = pk2(yi[k], yi[k]);
            zd[k] = pk2(zi[k], zi[k]);
            ax2[k] = ay2[k] = az2[k] = 0ull;
        }
        const int jb = J * TI;
        for (int sc = 0; sc < TI / SYM_SUB; ++sc) {
            const int buf = sc & 1;
#pragma unroll 1
            for (int q = 0; q < SYM_SUB / 64; ++q) {
                const int j0 = jb + sc * SYM_SUB + q * 64 + lane;
                const float4 pa = __ldg(fpos + j0), pb = __ldg(fpos + j0 + 32);
                f32x2 xj = pk2(pa.x, pb.x), yj = pk2(pa.y, pb.y), zj = pk2(pa.z, pb.z);
                f32x2 bx = 0ull, by = 0ull, bz = 0ull;
#pragma unroll 2
                for (int r = 0; r < 32; ++r) {
#pragma unroll
                    for (int k = 0; k < IPT; ++k) {
                        const f32x2 dx = sub2(xj, xd[k]), dy = sub2(yj, yd[k]), dz = sub2(zj, zd[k]);
                        const f32x2 c3 = CUT ? pair_c3x2_cut(dx, dy, dz, F.cut_s0, F.cut_inv_w) : pair_c3x2(dx, dy, dz);
                        ax2[k] = fma2(c3, dx, ax2[k]);
                        ay2[k] = fma2(c3, dy, ay2[k]);
                        az2[k] = fma2(c3, dz, az2[k]);
                        bx = fma2(c3, dx, bx);
                        by = fma2(c3, dy, by);
                        bz = fma2(c3, dz, bz);
                    }
                    xj = __shfl_sync(0xffffffffu, xj, src);
                    yj = __shfl_sync(0xffffffffu, yj, src);
                    zj = __shfl_sync(0xffffffffu, zj, src);
                    bx = __shfl_sync(0xffffffffu, bx, src);
                    by = __shfl_sync(0xffffffffu, by, src);
                    bz = __shfl_sync(0xffffffffu, bz, src);
                }
                float l0, h0;
                upk2(bx, l0, h0);
                s_acc[buf][0][w][q * 64 + lane] = l0;
                s_acc[buf][0][w][q * 64 + 32 + lane] = h0;
                upk2(by, l0, h0);
                s_acc[buf][1][w][q * 64 + lane] = l0;
                s_acc[buf][1][w][q * 64 + 32 + lane] = h0;
                upk2(bz, l0, h0);
                s_acc[buf][2][w][q * 64 + lane] = l0;
                s_acc[buf][2][w][q * 64 + 32 + lane] = h0;
            }
            // one barrier per combine step: the other buffer's readers (previous step)
            // finished before they reached it
            __syncthreads();
            for (int j = threadIdx.x; j < SYM_SUB; j += BT) {
                float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
                for (int ww = 0; ww < NW; ++ww) {
                    sx += s_acc[buf][0][ww][j];
                    sy += s_acc[buf][1][ww][j];
                    sz += s_acc[buf][2][ww][j];
                }
                fixed_add3(F.psum, F.psum_ld, jb + sc * SYM_SUB + j, -sx, -sy, -sz, F.qscale, F.err);
            }
        }
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            float l0, h0;
            upk2(ax2[k], l0, h0);
            ax[k] = l0 + h0;
            upk2(ay2[k], l0, h0);
            ay[k] = l0 + h0;
            upk2(az2[k], l0, h0);
            az[k] = l0 + h0;
        }
    }
#pragma unroll
    for (int k = 0; k < IPT; ++k)
        fixed_add3(F.psum, F.psum_ld, I * TI + k * BT + threadIdx.x, ax[k], ay[k], az[k], F.qscale, F.err);
}

// Dynamic unit queue: a persistent CTA takes the next unit index from sched[0] (the
// fixed-point sums are order-independent, so which CTA evaluates a unit changes no
// result); the last CTA to
// finish resets both words for the next launch on the stream.
__device__ __forceinline__ long long next_unit(unsigned long long* sched, long long& s_u)
{
    __syncthreads();  // every thread has read the previous index
    if (threadIdx.x == 0) s_u = (long long)atomicAdd(sched, 1ull);
    __syncthreads();
    return s_u;
}

__device__ __forceinline__ void leave_queue(unsigned long long* sched)
{
    if (threadIdx.x == 0 && atomicAdd(sched + 1, 1ull) == gridDim.x - 1) {
        sched[0] = 0ull;
        sched[1] = 0ull;
    }
}

// Persistent symmetric kernel on packed FP32 pairs: tile-pair units from the dynamic
// queue.  The 8-target variants are held to 128 registers (a few spills) for one more
// resident CTA per SM, which measured 1% faster than their natural 133.
template <int BT, int IPT>
__global__ void __launch_bounds__(BT, (IPT == 8 ? 65536 / (BT * 128) : 1))
    k_forces_sym2(const float4* __restrict__ fpos, ForceArgs F)
{
    constexpr int TI = BT * IPT;
    __shared__ float s_acc[2][3][BT / 32][SYM_SUB];
    __shared__ float4 sj[BT];
    __shared__ long long s_u;
    // tiles from the live count on hold only far-away dummies, whose terms with live ions
    // are exactly zero: units that reach such a tile (J >= I) are skipped.  The count is read again for every unit (a volatile load),
    // so that it takes no register across the unit's code, which sits at the register cap.
    for (;;) {
        const long long u = next_unit(F.sched, s_u);
        if (u >= F.U) break;
        int I, J;
        tri_unit(u, F.JS, I, J);
        if (F.n_live && J * TI >= *(volatile const int*)F.n_live) continue;
        sym2_unit<BT, IPT>(fpos, F, I, J, s_acc, sj);
    }
    leave_queue(F.sched);
}

// One (target tile t, source chunk c) unit written to partial slot c (batched launch,
// where every unit is its own task and a tile's W = JS slots are its chunks).
template <int BT, int IPT>
__device__ __forceinline__ void forces_unit(const float4* __restrict__ fpos, float4* __restrict__ part,
                                            const ForceArgs& F, int t, int c, float4* sj)
{
    float xi[IPT], yi[IPT], zi[IPT], ax[IPT], ay[IPT], az[IPT];
#pragma unroll
    for (int k = 0; k < IPT; ++k) {
        const float4 p = fpos[t * F.TI + k * BT + threadIdx.x];
        xi[k] = p.x;
        yi[k] = p.y;
        zi[k] = p.z;
        ax[k] = 0.f;
        ay[k] = 0.f;
        az[k] = 0.f;
    }
    const int j0 = c * F.JC;
    const int j1 = min(j0 + F.JC, F.n_pad);
    pair_chunk<BT, IPT>(fpos, j0, j1, xi, yi, zi, ax, ay, az, sj);
    float4* out = part + (long long)c * F.n_pad + t * F.TI + threadIdx.x;
#pragma unroll
    for (int k = 0; k < IPT; ++k) out[k * BT] = make_float4(ax[k], ay[k], az[k], 0.f);
}

}  // namespace od
