// Device code shared by the single-run kernels (od_kernels.cu) and the batched
// persistent kernel (od_batch.cu): helpers and the body of every phase of a step.
#pragma once

#include "od_internal.h"

namespace od {

// ------------------------------------------------------------------ helpers
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

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Philox4x32-10 (Salmon et al., SC'11): key = seed, counter = (id lo, id hi, word2, stream)
__device__ __forceinline__ uint4 philox(const Phys& P, unsigned long long id, uint32_t w2, uint32_t stream)
{
    uint4 c = make_uint4((uint32_t)id, (uint32_t)(id >> 32), w2, stream);
    uint32_t k0 = P.key0, k1 = P.key1;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// uniform in (0, 1): (w + 1/2) 2^-32
__device__ __forceinline__ double unif(uint32_t w) { return ((double)w + 0.5) * 2.3283064365386963e-10; }

__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, double& n0, double& n1)
{
    const double rad = sqrt(-2.0 * log(unif(a)));
    const double t = 6.283185307179586 * unif(b);
    double s, c;
    sincos(t, &s, &c);
    n0 = rad * c;
    n1 = rad * s;
}

__device__ __forceinline__ double ncdf(double z) { return 0.5 * erfc(-z * 0.70710678118654752); }
__device__ __forceinline__ double npdf(double z) { return exp(-0.5 * z * z) * 0.39894228040143268; }

// flux through the bottom face up to axial speed v: int_0^v v' N(v'; u, s^2) dv'
static __device__ double flux_bottom(double v, double u, double s)
{
    const double z = (v - u) / s, z0 = -u / s;
    return u * (ncdf(z) - ncdf(z0)) + s * (npdf(z0) - npdf(z));
}

// flux through the top face from axial speed v < 0 up to 0: -int_v^0 v' N(v'; u, s^2) dv'
static __device__ double flux_top(double v, double u, double s)
{
    const double z = (v - u) / s, z0 = -u / s;
    return -u * (ncdf(z0) - ncdf(z)) + s * (npdf(z0) - npdf(z));
}

// Invert a monotone flux CDF F on [lo, hi] for the value target: Newton steps on
// F(v) - target with derivative |v| N(v; u, s^2), kept inside a shrinking bracket
// (bisection when a step leaves it).
template <bool TOP>
__device__ double invert_flux(double target, double lo, double hi, double v, double u, double s)
{
    for (int it = 0; it < 100; ++it) {
        const double F = TOP ? flux_top(v, u, s) : flux_bottom(v, u, s);
        const double g = TOP ? (target - F) : (F - target);  // increasing in v
        if (g < 0) lo = v;
        else hi = v;
        const double dg = fabs(v) * npdf((v - u) / s) / s;
        // converged once the Newton correction is below ~1e-13 of the speed scale; the
        // check comes before the bracket test, which a sub-ulp step would fail
        const double tol = 1e-13 * fmax(fabs(v), s);
        if (dg > 0) {
            const double step = g / dg;
            if (fabs(step) <= tol) {
                v -= step;
                break;
            }
        }
        double vn = dg > 0 ? v - g / dg : 0.5 * (lo + hi);
        if (!(vn > lo && vn < hi)) vn = 0.5 * (lo + hi);
        v = vn;
        if (hi - lo <= tol) break;
    }
    return v;
}

// App. B: face by flux probability, position uniform on the face, flux-weighted velocity
static __device__ void sample_injection(const Phys& P, unsigned long long id, uint32_t sn, Inj& o)
{
    const uint4 A = philox(P, id, sn, ST_INJ_A);
    const uint4 Bw = philox(P, id, sn, ST_INJ_B);
    double n0, n1;
    box_muller(Bw.x, Bw.y, n0, n1);
    if ((unsigned long long)A.x < P.Tbt) {
        const int f = (unsigned long long)A.x < P.Tb ? 0 : 1;
        const double rho = P.R * sqrt(unif(A.y));
        double s, c;
        sincos(6.283185307179586 * unif(A.z), &s, &c);
        o.x = rho * c;
        o.y = rho * s;
        o.z = f == 0 ? -0.5 * P.H : 0.5 * P.H;
        o.vx = P.sig * n0;
        o.vy = P.sig * n1;
        // flux-weighted axial speed: the tabulated inverse CDF brackets the root and gives
        // the starting point, Newton polishes it to ~1e-13 (FP64 is slow on this GPU: a
        // few iterations instead of a bisection from the whole range)
        const double U = unif(A.w);
        const double xk = U * VTAB_K;
        const int k = min((int)xk, VTAB_K - 1);
        const double* tab = P.vtab + (f == 0 ? 0 : VTAB_K + 1);
        const double t0 = tab[k], t1 = tab[k + 1];
        const double pad = 1e-12 * fmax(fmax(fabs(t0), fabs(t1)), P.sig);
        const double v0 = t0 + (xk - k) * (t1 - t0);
        if (f == 0)
            o.vz = invert_flux<false>(U * P.gmax_b, fmax(fmin(t0, t1) - pad, 0.0), fmax(t0, t1) + pad, v0, P.u, P.sig);
        else
            o.vz = invert_flux<true>(U * P.gmax_t, fmin(t0, t1) - pad, fmin(fmax(t0, t1) + pad, 0.0), v0, P.u, P.sig);
        o.face = f;
    } else {
        double s, c;
        sincos(6.283185307179586 * unif(A.y), &s, &c);
        o.x = P.R * c;
        o.y = P.R * s;
        o.z = P.H * (unif(A.z) - 0.5);
        const double vr = P.sig * sqrt(-2.0 * log(unif(A.w)));  // Rayleigh: flux-weighted radial speed
        const double vt = (P.flags & OD_F_PAPER_SIDE) ? 0.0 : P.sig * n0;
        o.vx = -vr * c - vt * s;
        o.vy = -vr * s + vt * c;
        o.vz = P.u + P.sig * n1;
        o.face = 2;
    }
    o.id = id;
}

// E_out = -grad P (App. A): E = (-x G, -y G, -z K), G and K over monomials r2^p z2^q, p+q <= 3
__device__ __forceinline__ void eout_field(const Phys& P, double x, double y, double z, double& ex, double& ey,
                                           double& ez)
{
    const double r2 = x * x + y * y, z2 = z * z;
    const double r4 = r2 * r2, z4 = z2 * z2;
    const double m[10] = {1.0, r2, z2, r4, r2 * z2, z4, r4 * r2, r4 * z2, r2 * z4, z4 * z2};
    double G = 0.0, K = 0.0;
#pragma unroll
    for (int t = 0; t < 10; ++t) {
        G += P.Gc[t] * m[t];
        K += P.Kc[t] * m[t];
    }
    ex = -x * G;
    ey = -y * G;
    ez = -z * K;
}

__device__ __forceinline__ float4 scaled(const Phys& P, double x, double y, double z, double ls_inv)
{
    return make_float4((float)(x * ls_inv), (float)(y * ls_inv), (float)(z * ls_inv), 0.0f);
}

__device__ __forceinline__ double rnd32(double v) { return (double)(float)v; }

// Number of superions injected in step sn under the flux rule: Poisson with mean lam,
// split into chunks of at most 64, each drawn by inversion (summing e^-l l^x / x! in
// increasing x until the sum reaches one uniform); uniform j of the step is word j mod 4
// of the Philox block with counter (j / 4, 0, sn, ST_INJ_N).  FP64 throughout.
__device__ __forceinline__ int poisson_injections(const Phys& P, uint32_t sn)
{
    double rem = P.inj_lambda;
    int k = 0;
    for (int j = 0; rem > 0.0; ++j) {
        const double l = rem > 64.0 ? 64.0 : rem;
        rem -= l;
        const uint4 w = philox(P, (unsigned long long)(j >> 2), sn, ST_INJ_N);
        const uint32_t wj = (j & 3) == 0 ? w.x : (j & 3) == 1 ? w.y : (j & 3) == 2 ? w.z : w.w;
        const double U = unif(wj);
        double pr = exp(-l), F = pr;
        int x = 0;
        while (U > F && x < 100000) {
            ++x;
            pr = pr * (l / (double)x);
            F += pr;
        }
        k += x;
    }
    return k;
}

// ------------------------------------------------- push + scan + compaction
constexpr int PUSH_BT = 256;

constexpr unsigned FLAG_A = 1u, FLAG_P = 2u;

__device__ __forceinline__ unsigned long long pack_status(uint32_t epoch, unsigned flag, int val)
{
    return ((unsigned long long)epoch << 32) | ((unsigned long long)flag << 30) | (unsigned long long)(val & 0x3fffffff);
}

// One scan tile: given_tile >= 0 names the tile (batched launch, tiles of a run handed
// out in order); otherwise the tile id comes from the run's launch-order counter.
template <int BT>
__device__ __forceinline__ void push_scan_body(const Phys& P, const Bufs& B, int n_tiles, double ls_inv, int given_tile)
{
    __shared__ unsigned s_tile;
    __shared__ int s_wsum[BT / 32];
    __shared__ int s_total, s_prefix, s_last, s_m, s_k;
    __shared__ int s_face[3];
    Ctrl* C = B.ctrl;
    const long long step = C->step;
    const int src = (int)(step & 1), dst = src ^ 1;
    const uint32_t sn = (uint32_t)(step + 1);
    const long long cap = B.cap;
    const bool flux = (P.flags & OD_F_FLUX_INJECT) != 0;
    // ions alive at the start of the step (only the last tile, after every other tile
    // has finished, writes the new count)
    const int n_live = *(volatile int*)&C->n_cur;
    if (threadIdx.x == 0) s_tile = given_tile >= 0 ? (unsigned)given_tile : atomicAdd(&C->tile_counter, 1u);
    __syncthreads();
    const int tile = (int)s_tile;
    const int i = tile * BT + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    double x = 0, y = 0, z = 0, vx = 0, vy = 0, vz = 0;
    unsigned long long id = 0;
    int cls = -2;  // -2 stays, -1 outflow, k >= 0 absorbed by grain k
    if (i < n_live) {
        const double* X = B.x[src];
        const double* V = B.v[src];
        x = X[i];
        y = X[cap + i];
        z = X[2 * cap + i];
        vx = V[i];
        vy = V[cap + i];
        vz = V[2 * cap + i];
        id = B.id[src][i];
        const float4 a = B.acc[i];
        const double h = 0.5 * P.dt;
        vx += h * (double)a.x;
        vy += h * (double)a.y;
        vz += h * (double)a.z;
        if (P.flags & OD_F_FP32_STATE) vx = rnd32(vx), vy = rnd32(vy), vz = rnd32(vz);
        x += P.dt * vx;
        y += P.dt * vy;
        z += P.dt * vz;
        if (P.flags & OD_F_FP32_STATE) x = rnd32(x), y = rnd32(y), z = rnd32(z);
        if (!isfinite(x + y + z + vx + vy + vz)) atomicOr(&C->err, ERR_NAN);
        if (!(P.flags & OD_F_NO_ABSORB)) {
            for (int k = 0; k < P.D; ++k) {
                const double dx = x - P.gx[k], dy = y - P.gy[k], dz = z - P.gz[k];
                const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                if (d2 <= P.ga2[k]) {
                    cls = k;
                    break;
                }
            }
        }
        if (cls == -2 && !(P.flags & OD_F_NO_BOUNDARY)) {
            const double r2 = __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y));
            if (r2 > P.R2 || fabs(z) > P.hz) cls = -1;
        }
    }
    const int removed = cls != -2;

    // event counts with one atomic per warp
    const unsigned bo = __ballot_sync(0xffffffffu, cls == -1);
    if (lane == 0 && bo) atomicAdd(&C->ev_step[8], __popc(bo));
    for (int k = 0; k < P.D; ++k) {
        const unsigned bk = __ballot_sync(0xffffffffu, cls == k);
        if (lane == 0 && bk) atomicAdd(&C->ev_step[k], __popc(bk));
    }

    // block-wide exclusive scan of the removal flags
    const unsigned bal = __ballot_sync(0xffffffffu, removed);
    const int wrank = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) s_wsum[warp] = __popc(bal);
    __syncthreads();
    if (warp == 0) {
        const int v = lane < BT / 32 ? s_wsum[lane] : 0;
        int inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane < BT / 32) s_wsum[lane] = inc - v;
        if (lane == BT / 32 - 1) s_total = inc;
    }
    __syncthreads();
    const int lrank = s_wsum[warp] + wrank;

    // decoupled look-back across tiles (tile ids are taken in launch order, so every
    // predecessor is running or done); the wait is bounded and reports ERR_TIMEOUT
    // warp 0 probes 32 predecessors per read: lane l looks at tile base - l
    if (warp == 0) {
        const int total = s_total;
        unsigned long long* st = B.tile_status;
        int excl = 0;
        if (tile == 0) {
            // (the wait self-test withholds tile 0's prefix so that its successors time out)
            if (lane == 0 && !P.test_hold_tile0) st_release_u64(st, pack_status(sn, FLAG_P, total));
        } else {
            if (lane == 0) st_release_u64(st + tile, pack_status(sn, FLAG_A, total));
            int base = tile - 1;
            long long spins = 0;
            unsigned ns = 32;
            while (true) {
                const int t = base - lane;
                unsigned fl = FLAG_P;  // before tile 0: an inclusive prefix of zero
                int val = 0;
                if (t >= 0) {
                    const unsigned long long w = ld_acquire_u64(st + t);
                    fl = (uint32_t)(w >> 32) == sn ? (unsigned)(w >> 30) & 3u : 0u;
                    val = (int)(w & 0x3fffffffull);
                }
                const unsigned pmask = __ballot_sync(0xffffffffu, fl == FLAG_P);
                const unsigned zmask = __ballot_sync(0xffffffffu, fl == 0u);
                const int first_p = pmask ? __ffs(pmask) - 1 : 32;  // nearest inclusive prefix
                const unsigned need = first_p >= 31 ? 0xffffffffu : ((1u << (first_p + 1)) - 1u);
                if (zmask & need) {  // a tile up to that prefix has not published yet
                    if (++spins > P.spin_limit) {
                        if (lane == 0) atomicOr(&C->err, ERR_TIMEOUT);
                        break;
                    }
                    __nanosleep(ns);
                    if (ns < 1024) ns *= 2;
                    continue;
                }
                int contrib = lane <= first_p ? val : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) contrib += __shfl_down_sync(0xffffffffu, contrib, o);
                excl += __shfl_sync(0xffffffffu, contrib, 0);
                if (first_p < 32) break;
                base -= 32;
            }
            if (lane == 0) st_release_u64(st + tile, pack_status(sn, FLAG_P, excl + total));
        }
        if (lane == 0) {
            // keep destinations in bounds even if a wait gave up
            if (excl > tile * BT) excl = tile * BT;
            if (excl < 0) excl = 0;
            s_prefix = excl;
            atomicAdd(&C->removed_total, total);
        }
    }
    __syncthreads();
    const int prefix = s_prefix;

    if (i < n_live) {
        if (!removed) {
            const int d = i - prefix - lrank;  // stable compaction
            double* X = B.x[dst];
            double* V = B.v[dst];
            X[d] = x;
            X[cap + d] = y;
            X[2 * cap + d] = z;
            V[d] = vx;
            V[cap + d] = vy;
            V[2 * cap + d] = vz;
            B.id[dst][d] = id;
            B.fpos[d] = scaled(P, x, y, z, ls_inv);
        } else {
            const int r = prefix + lrank;  // global rank among removed ions, index order
            Rem rm;
            rm.vx = vx;
            rm.vy = vy;
            rm.vz = vz;
            rm.cls = cls;
            rm.pad = 0;
            B.rem[r] = rm;
            if (!flux) {  // 1:1 replacement: the removed ion's thread samples its successor
                Inj in;
                sample_injection(P, C->next_id + (unsigned long long)r, sn, in);
                if (P.flags & OD_F_FP32_STATE) {
                    in.x = rnd32(in.x), in.y = rnd32(in.y), in.z = rnd32(in.z);
                    in.vx = rnd32(in.vx), in.vy = rnd32(in.vy), in.vz = rnd32(in.vz);
                }
                in.pad = 0;
                B.inj[r] = in;
            }
        }
    }

    // the last tile to finish places the injected ions at the end, in rank order
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&C->done_counter, 1u) == (unsigned)(n_tiles - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x < 3) s_face[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        int m = *(volatile int*)&C->removed_total;
        if (m > n_live) m = n_live;
        s_m = m;
        // injections: one per removed ion, or a Poisson number from the fluxes (clamped
        // to the capacity, which reports an overflow)
        int k = flux ? poisson_injections(P, sn) : m;
        if (n_live - m + k > P.N) {
            k = P.N - (n_live - m);
            atomicOr(&C->err, ERR_OVERFLOW);
        }
        s_k = k;
    }
    __syncthreads();
    const int m = s_m, kin = s_k;
    for (int r = threadIdx.x; r < kin; r += BT) {
        double ix, iy, iz, ivx, ivy, ivz;
        unsigned long long iid;
        int face;
        if (flux) {
            Inj in;
            sample_injection(P, C->next_id + (unsigned long long)r, sn, in);
            if (P.flags & OD_F_FP32_STATE) {
                in.x = rnd32(in.x), in.y = rnd32(in.y), in.z = rnd32(in.z);
                in.vx = rnd32(in.vx), in.vy = rnd32(in.vy), in.vz = rnd32(in.vz);
            }
            ix = in.x, iy = in.y, iz = in.z, ivx = in.vx, ivy = in.vy, ivz = in.vz, iid = in.id, face = in.face;
        } else {
            const Inj* in = B.inj + r;
            ix = __ldcg(&in->x), iy = __ldcg(&in->y), iz = __ldcg(&in->z);
            ivx = __ldcg(&in->vx), ivy = __ldcg(&in->vy), ivz = __ldcg(&in->vz);
            iid = __ldcg(&in->id);
            face = __ldcg(&in->face);
        }
        const int d = n_live - m + r;
        double* X = B.x[dst];
        double* V = B.v[dst];
        X[d] = ix;
        X[cap + d] = iy;
        X[2 * cap + d] = iz;
        V[d] = ivx;
        V[cap + d] = ivy;
        V[2 * cap + d] = ivz;
        B.id[dst][d] = iid;
        B.fpos[d] = scaled(P, ix, iy, iz, ls_inv);
        atomicAdd(&s_face[face], 1);
    }
    // slots vacated when fewer ions entered than left: far-away dummies for the pair kernel
    const int n_new = n_live - m + kin;
    for (int d = n_new + threadIdx.x; d < n_live; d += BT) {
        const float far = 3.0e4f + 7.0f * (float)(d - n_new);
        B.fpos[d] = make_float4(far, far, far, 0.0f);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        C->ev_step[9] += s_face[0];
        C->ev_step[10] += s_face[1];
        C->ev_step[11] += s_face[2];
        C->next_id += (unsigned long long)kin;
        C->n_cur = n_new;
        C->tile_counter = 0u;
        C->done_counter = 0u;
    }
}

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
// in row-major order, split into contiguous ranges over the persistent blocks.
//
// Unit (I, J > I): warp w holds 32 IPT targets of tile I (IPT per lane) and walks tile J
// in groups of 32 sources, one per lane.  Each source travels round the warp by shuffles
// together with its own accumulator, so after 32 rotations every lane has met every
// source of the group and each accumulator is back on its lane.  The source-side sums of
// the warps are combined in shared memory in a fixed warp order, SUB sources at a time
// (double buffered, one barrier per SUB sources).
// Unit (I, I): the ordered pairs of the tile through pair_chunk (the self pair is 0).
//
// Partial slots (deterministic, each written exactly once per evaluation): the target-
// side sum of unit (I, J) goes to slot J of the ions of tile I, its source-side sum to
// slot I of the ions of tile J, and unit (I, I) fills slot I of tile I.  Every ion has
// T slots, summed by the kick.
template <int BT, int IPT>
__global__ void __launch_bounds__(BT) k_forces_sym(const float4* __restrict__ fpos, float4* __restrict__ part,
                                                   ForceArgs F)
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
                    part[(long long)I * F.n_pad + jb + sc * SUB + j] = make_float4(sx, sy, sz, 0.f);
                }
            }
        }
        float4* out = part + (long long)J * F.n_pad + I * TI + threadIdx.x;
#pragma unroll
        for (int k = 0; k < IPT; ++k) out[k * BT] = make_float4(ax[k], ay[k], az[k], 0.f);
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

// pair_c3_cut for two pairs at once: the packed plain coefficient's steps, then the
// switching bracket per lane
__device__ __forceinline__ f32x2 pair_c3x2_cut(f32x2 dx, f32x2 dy, f32x2 dz, float s0, float w_inv)
{
    const f32x2 eps2 = pk2(1e-24f, 1e-24f);
    f32x2 r2 = fma2(dx, dx, eps2);
    r2 = fma2(dy, dy, r2);
    r2 = fma2(dz, dz, r2);
    float ra, rb;
    upk2(r2, ra, rb);
    const float ria = rsqrt_approx(ra), rib = rsqrt_approx(rb);
    const f32x2 ri = pk2(ria, rib);
    float sa, sb;
    upk2(mul2(r2, ri), sa, sb);
    const f32x2 e = pk2(ex2_approx(-sa), ex2_approx(-sb));
    const f32x2 br = pk2(switch_bracket(sa, ria, s0, w_inv), switch_bracket(sb, rib, s0, w_inv));
    return mul2(mul2(e, mul2(ri, ri)), br);
}

constexpr int SYM_SUB = 128;  // sources per combine step of the symmetric kernels

// One tile-pair unit (I, J >= I) of the symmetric kernel with packed FP32 pairs: the same
// units, slots and fixed combine order as k_forces_sym, but the travelling packet holds
// two sources (the lane's sources q*64 + lane and q*64 + 32 + lane of the group), each
// target is duplicated into both halves of a pair, and every FP32 operation of the pair
// term acts on the two sources in one instruction.  Source-side sums are accumulated
// with the target-side sign and negated when the warps' sums are combined.  Every unit
// starts on combine buffer 0 and ends on buffer 1, so consecutive units need no barrier
// between them beyond the one per combine step.
// slot_i / slot_j: the partial slots that receive the sums of the ions of tile I / J (the
// all-pairs kernels pass J / I; the cutoff passes the positions of J and I in the other
// tile's neighbour list)
template <int BT, int IPT, bool CUT = false>
__device__ __forceinline__ void sym2_unit(const float4* __restrict__ fpos, float4* __restrict__ part,
                                          const ForceArgs& F, int I, int J, float (&s_acc)[2][3][BT / 32][SYM_SUB],
                                          float4* sj, int slot_i, int slot_j)
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
                part[(long long)slot_j * F.n_pad + jb + sc * SYM_SUB + j] = make_float4(-sx, -sy, -sz, 0.f);
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
    float4* out = part + (long long)slot_i * F.n_pad + I * TI + threadIdx.x;
#pragma unroll
    for (int k = 0; k < IPT; ++k) out[k * BT] = make_float4(ax[k], ay[k], az[k], 0.f);
}

// Persistent symmetric kernel on packed FP32 pairs: contiguous ranges of tile-pair units.
// The 8-target variants are held to 128 registers (a few spills) for one more resident
// CTA per SM, which measured 1% faster than their natural 133.
template <int BT, int IPT>
__global__ void __launch_bounds__(BT, (IPT == 8 ? 65536 / (BT * 128) : 1)) k_forces_sym2(const float4* __restrict__ fpos, float4* __restrict__ part,
                                                    ForceArgs F)
{
    __shared__ float s_acc[2][3][BT / 32][SYM_SUB];
    __shared__ float4 sj[BT];
    long long u = (long long)blockIdx.x * F.U / F.G;
    const long long u_end = (long long)(blockIdx.x + 1) * F.U / F.G;
    if (u >= u_end) return;
    int I, J;
    tri_unit(u, F.JS, I, J);
    for (; u < u_end; ++u) {
        sym2_unit<BT, IPT>(fpos, part, F, I, J, s_acc, sj, J, I);
        if (++J == F.JS) J = ++I;
    }
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

// ---------------------------------------------- kick, collisions, grain sums
constexpr int KICK_BT = 64;  // small blocks spread small runs over many SMs (FP64 is slow)

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// mode 0: after the push (second half kick + collisions); mode 1: forces only (creation
// or a replaced ion state)
template <int BT>
__device__ __forceinline__ void kick_body(const Phys& P, const Bufs& B, const ForceArgs& F, int mode, int blk)
{
    __shared__ double s_red[BT / 32][3];
    Ctrl* C = B.ctrl;
    const long long step = C->step;
    const int buf = mode == 0 ? (int)((step + 1) & 1) : (int)(step & 1);
    const uint32_t sn = (uint32_t)(step + 1);
    const int i = blk * BT + threadIdx.x;
    const bool live = i < C->n_cur;
    const long long cap = B.cap;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double x = 0, y = 0, z = 0;
    int coll = 0;
    if (live) {
        const double* X = B.x[buf];
        x = X[i];
        y = X[cap + i];
        z = X[2 * cap + i];
        float ax = 0.f, ay = 0.f, az = 0.f;
        if (!(P.flags & OD_F_NO_IONION)) {
            // slots of this ion: the blocks that covered its tile (ordered-pair kernel), one
            // per tile (symmetric kernel) or one per neighbour of the tile that holds its
            // sorted position (cutoff: slots 0 .. degree - 1)
            int ns = F.W;
            int q = i;  // position in the pair kernel's ion order
            if (F.cut) {
                q = F.rank[i];
                const int t = q / F.TI;
                ns = F.nbr_start[t + 1] - F.nbr_start[t];
            } else if (!F.sym) {
                const int t = i / F.TI;
                const long long u0 = (long long)t * F.JS;
                ns = owner_of(u0 + F.JS - 1, F.U, F.G) - owner_of(u0, F.U, F.G) + 1;
            }
            // blocked sum over the slots (up to ~1000 with the symmetric kernel)
            for (int s0 = 0; s0 < ns; s0 += 16) {
                const int s1 = min(ns, s0 + 16);
                float bx = 0.f, by = 0.f, bz = 0.f;
#pragma unroll 8
                for (int s = s0; s < s1; ++s) {
                    const float4 p = __ldcs(B.part + (long long)s * F.n_pad + q);
                    bx += p.x;
                    by += p.y;
                    bz += p.z;
                }
                ax += bx;
                ay += by;
                az += bz;
            }
            ax *= -P.k_ii;
            ay *= -P.k_ii;
            az *= -P.k_ii;
        }
        // bare Coulomb force of the grains (asymmetric model): FP32 terms from FP64
        // separations, like the pair forces
        for (int k = 0; k < P.D; ++k) {
            const float dx = (float)(x - P.gx[k]), dy = (float)(y - P.gy[k]), dz = (float)(z - P.gz[k]);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float ri = rsqrt_approx(r2);
            const float c = (float)(P.kdi * C->Q[k]) * (ri * ri * ri);
            ax = fmaf(c, dx, ax);
            ay = fmaf(c, dy, ay);
            az = fmaf(c, dz, az);
        }
        // E_out (FP64 polynomial) and the driving field
        double bx = 0.0, by = 0.0, bz = P.qm * P.E;
        if (P.eout) {
            double ex, ey, ez;
            eout_field(P, x, y, z, ex, ey, ez);
            bx += P.qm * ex;
            by += P.qm * ey;
            bz += P.qm * ez;
        }
        const float4 a = make_float4((float)((double)ax + bx), (float)((double)ay + by), (float)((double)az + bz), 0.f);
        B.acc[i] = a;
        if (mode == 0) {
            double* V = B.v[buf];
            double vx = V[i], vy = V[cap + i], vz = V[2 * cap + i];
            const double h = 0.5 * P.dt;
            vx += h * (double)a.x;
            vy += h * (double)a.y;
            vz += h * (double)a.z;
            // Andersen collision with the neutrals: integer threshold on a Philox word
            const unsigned long long id = B.id[buf][i];
            const uint4 w = philox(P, id, sn, ST_COLL);
            if ((unsigned long long)w.x < P.Tcoll) {
                const uint4 wv = philox(P, id, sn, ST_COLL_VEL);
                double n0, n1, n2, n3;
                box_muller(wv.x, wv.y, n0, n1);
                box_muller(wv.z, wv.w, n2, n3);
                vx = P.sig_n * n0;
                vy = P.sig_n * n1;
                vz = P.sig_n * n2;
                coll = 1;
            }
            if (P.flags & OD_F_FP32_STATE) vx = rnd32(vx), vy = rnd32(vy), vz = rnd32(vz);
            V[i] = vx;
            V[cap + i] = vy;
            V[2 * cap + i] = vz;
        }
    }
    const unsigned bc = __ballot_sync(0xffffffffu, coll);
    if (lane == 0 && bc) atomicAdd(&C->ev_step[12], __popc(bc));

    // grain side of Eq. 1 without the prefactor q Q_k / (4 pi eps0):
    // sum_i (1 + rho/lambda) exp(-rho/lambda) (r_k - r_i) / rho^3; FP32 terms from FP64
    // separations, FP64 sums in a fixed order (warp tree, then block tree)
    const float lam_inv = (float)P.lam_inv;
    const float lam_inv_l2 = (float)(P.lam_inv * 1.4426950408889634);
    for (int k = 0; k < P.D; ++k) {
        double fx = 0.0, fy = 0.0, fz = 0.0;
        if (live) {
            const float dx = (float)(P.gx[k] - x), dy = (float)(P.gy[k] - y), dz = (float)(P.gz[k] - z);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float ri = rsqrt_approx(r2);
            const float rho = r2 * ri;
            const float f = fmaf(rho, lam_inv, 1.0f) * ex2_approx(-rho * lam_inv_l2) * (ri * ri * ri);
            fx = (double)(f * dx);
            fy = (double)(f * dy);
            fz = (double)(f * dz);
        }
        fx = warp_sum(fx);
        fy = warp_sum(fy);
        fz = warp_sum(fz);
        if (lane == 0) {
            s_red[warp][0] = fx;
            s_red[warp][1] = fy;
            s_red[warp][2] = fz;
        }
        __syncthreads();
        if (warp == 0) {
            double a0 = lane < BT / 32 ? s_red[lane][0] : 0.0;
            double a1 = lane < BT / 32 ? s_red[lane][1] : 0.0;
            double a2 = lane < BT / 32 ? s_red[lane][2] : 0.0;
            a0 = warp_sum(a0);
            a1 = warp_sum(a1);
            a2 = warp_sum(a2);
            if (lane == 0) {
                double* o = B.dpart + ((long long)blk * MAXD + k) * 3;
                o[0] = a0;
                o[1] = a1;
                o[2] = a2;
            }
        }
        __syncthreads();
    }
}

// --------------------------------------------------------------- grain tail
constexpr int DUST_BT = 256;

__device__ __forceinline__ void dust_body(const Phys& P, const Bufs& B, int nb, int mode)
{
    __shared__ double s_S[MAXD][3];
    __shared__ double s_rec[MAXD][REC];
    Ctrl* C = B.ctrl;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // deterministic reduction of the kick kernel's per-block grain sums: warp w takes
    // component pairs w, w+8, ...; lanes stride the blocks, then a fixed shuffle tree
    for (int pc = warp; pc < P.D * 3; pc += DUST_BT / 32) {
        const int k = pc / 3, c = pc % 3;
        double s = 0.0;
        for (int b = lane; b < nb; b += 32) s += B.dpart[((long long)b * MAXD + k) * 3 + c];
        s = warp_sum(s);
        if (lane == 0) s_S[k][c] = s;
    }
    __syncthreads();
    const int k = threadIdx.x;
    if (k < P.D) {
        const double Q = C->Q[k];
        double ex = 0.0, ey = 0.0, ez = 0.0;
        if (P.eout) eout_field(P, P.gx[k], P.gy[k], P.gz[k], ex, ey, ez);
        const double c = P.korb * Q;
        const double fo[3] = {c * s_S[k][0] + ex * Q, c * s_S[k][1] + ey * Q, c * s_S[k][2] + ez * Q};
        for (int j = 0; j < 3; ++j) C->f_orbit[k][j] = fo[j];
        if (mode == 0) {
            // Eq. 2: Coulomb force of the other grains
            double fdd[3] = {0.0, 0.0, 0.0};
            for (int p = 0; p < P.D; ++p) {
                if (p == k) continue;
                const double dx = P.gx[k] - P.gx[p], dy = P.gy[k] - P.gy[p], dz = P.gz[k] - P.gz[p];
                const double d = sqrt(dx * dx + dy * dy + dz * dz);
                const double cc = P.inv4pieps0 * Q * C->Q[p] / (d * d * d);
                fdd[0] += cc * dx;
                fdd[1] += cc * dy;
                fdd[2] += cc * dz;
            }
            // Eq. 3: momentum of the ions absorbed this step, summed in index order
            const int m = C->removed_total;
            double pm[3] = {0.0, 0.0, 0.0};
            for (int r = 0; r < m; ++r) {
                const Rem rm = B.rem[r];
                if (rm.cls == k) {
                    pm[0] += P.m * rm.vx;
                    pm[1] += P.m * rm.vy;
                    pm[2] += P.m * rm.vz;
                }
            }
            for (int j = 0; j < 3; ++j) {
                s_rec[k][1 + j] = fo[j];
                s_rec[k][4 + j] = fdd[j];
                s_rec[k][7 + j] = pm[j] / P.dt;
            }
            s_rec[k][10] = 0.0;
            s_rec[k][11] = 0.0;
            s_rec[k][12] = Q * P.E;  // Eq. 4
        }
    }
    __syncthreads();
    if (mode != 0) return;
    const long long step = C->step;
    const long long sn = step + 1;
    if (k < P.D) {
        double Q = C->Q[k];
        if (P.charge_model == OD_Q_CONSISTENT) {
            // absorbed superions plus the OML electron flux at the isolated-sphere potential
            const double a = P.ga[k];
            const double xe = Q * P.inv4pieps0 / a * P.e_over_kTe;
            const double fac = xe <= 0.0 ? exp(xe) : 1.0 + xe;
            const double flux = 4.0 * 3.141592653589793 * a * a * P.Ie0 * fac;
            Q = Q + P.q * (double)C->ev_step[k] - 1.602176634e-19 * flux * P.dt;
            C->Q[k] = Q;
        }
        s_rec[k][0] = Q;
        if (step < C->series_cap) {
            double* o = C->series + (step * MAXD + k) * REC;
            for (int j = 0; j < REC; ++j) o[j] = s_rec[k][j];
        }
        if (sn >= P.avg_start)
            for (int j = 0; j < REC; ++j) C->wsum[k][j] += s_rec[k][j];
    }
    __syncthreads();
    // one thread per event counter: record, accumulate, reset for the next step
    const int j = threadIdx.x;
    if (j < EV) {
        const int e = C->ev_step[j];
        if (step < C->series_cap) C->evseries[step * EV + j] = e;
        C->counters[j] += e;
        C->ev_step[j] = 0;
    } else if (j == 32) {
        C->counters[13] = sn;
        C->counters[14] = C->n_cur;
        C->counters[15] = (long long)C->next_id;
        if (sn >= P.avg_start) C->wcount += 1;
        C->removed_total = 0;
        C->step = sn;
    }
}

// window means and batch-means standard errors (20 batches) of every record entry
}  // namespace od
