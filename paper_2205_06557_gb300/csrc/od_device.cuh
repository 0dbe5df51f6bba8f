// Device code shared by the single-run kernels (od_kernels.cu) and the batched
// persistent kernel (od_batch.cu): helpers and the body of every phase of a step (the
// pair forces in od_pairs.cuh).
#pragma once

#include "od_internal.h"
#include "od_pairmath.cuh"

namespace od {

// ------------------------------------------------------------------ helpers

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

// Invert a monotone App. B flux CDF on [lo, hi] for the value target: Newton steps with
// derivative |v| N(v; u, s^2), kept inside a shrinking bracket (bisection when a step
// leaves it).  The bottom face's flux up to axial speed v is
//   int_0^v v' N(v'; u, s^2) dv' = u (Phi(z) - Phi(z0)) + s (phi(z0) - phi(z)),
// the top face's from v < 0 up to 0 is -u (Phi(z0) - Phi(z)) + s (phi(z0) - phi(z)), with
// z = (v - u) / s, z0 = -u / s (Phi, phi the standard normal CDF and density); Phi(z0)
// and phi(z0) are evaluated once per sample, Phi(z) and phi(z) once per iteration.
template <bool TOP>
__device__ double invert_flux(double target, double lo, double hi, double v, double u, double s)
{
    const double z0 = -u / s, c0 = ncdf(z0), p0 = npdf(z0);
    for (int it = 0; it < 100; ++it) {
        const double z = (v - u) / s;
        const double cz = ncdf(z), pz = npdf(z);
        const double F = TOP ? -u * (c0 - cz) + s * (p0 - pz) : u * (cz - c0) + s * (p0 - pz);
        const double g = TOP ? (target - F) : (F - target);  // increasing in v
        if (g < 0) lo = v;
        else hi = v;
        const double dg = fabs(v) * pz / s;
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

// The App. B sample of the ion with this id entering in step sn: computed ahead (during
// the previous step, beside the pair forces) when it is there, else now.  A sample is a
// function of (seed, id, sn) and the run's constants only, so both give the same bits.
static __device__ __forceinline__ void injection_for(const Phys& P, const Bufs& B, const Ctrl* C,
                                                     unsigned long long base, int r, uint32_t sn, Inj& o)
{
    if (r < C->ahead_n && C->ahead_base == base && C->ahead_sn == (long long)sn) {
        const Inj* a = B.inj_ahead + r;
        o.x = __ldcg(&a->x), o.y = __ldcg(&a->y), o.z = __ldcg(&a->z);
        o.vx = __ldcg(&a->vx), o.vy = __ldcg(&a->vy), o.vz = __ldcg(&a->vz);
        o.id = __ldcg(&a->id);
        o.face = __ldcg(&a->face);
    } else {
        sample_injection(P, base + (unsigned long long)r, sn, o);
    }
}

// Andersen collision: a zero-mean Maxwellian velocity at the neutral temperature
__device__ __forceinline__ void collision_velocity(const Phys& P, unsigned long long id, uint32_t sn, double& vx,
                                                   double& vy, double& vz)
{
    const uint4 wv = philox(P, id, sn, ST_COLL_VEL);
    double n0, n1, n2, n3;
    box_muller(wv.x, wv.y, n0, n1);
    box_muller(wv.z, wv.w, n2, n3);
    vx = P.sig_n * n0;
    vy = P.sig_n * n1;
    vz = P.sig_n * n2;
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

// ------------------------------------------------ close-pair cell lists
// The pair kernels see positions rounded to FP32 (scaled units s), which moves a pair's
// separation d by up to ~|s| 2^-24 and its 1/d^2 term by three times that relative to d:
// for the rare pairs much closer than the mean spacing this is the dominant error of an
// ion's force.  Every live ion is entered, at the end of the push (or whenever the FP32
// positions are rewritten), into a hashed grid of cells a little wider than twice the
// correction distance; the kick walks the 2 x 2 x 2 cells nearest to each ion (which
// hold every ion within that distance) and replaces the FP32-position value of every
// pair closer than it by its FP64 value.
// A bucket word is (epoch << 32) | first ion; entries of another epoch read as empty, so
// the grid is never cleared.  Ctrl::cp_epoch is the epoch of the last complete build
// (the one the kick reads); a build enters its ions under the next epoch and publishes it
// when it is complete, so no two builds share an epoch.
__device__ __forceinline__ int cp_cell(float s, float hinv) { return __float2int_rd(s * hinv); }

__device__ __forceinline__ unsigned cp_bucket(int cx, int cy, int cz, unsigned mask)
{
    return ((unsigned)cx * 73856093u ^ (unsigned)cy * 19349663u ^ (unsigned)cz * 83492791u) & mask;
}

__device__ __forceinline__ unsigned cp_next_epoch(unsigned e) { return e + 1u == 0u ? 1u : e + 1u; }

__device__ __forceinline__ void cp_insert(unsigned long long* head, int* next, unsigned mask, float hinv, unsigned epoch,
                                          int d, float4 f)
{
    const unsigned b = cp_bucket(cp_cell(f.x, hinv), cp_cell(f.y, hinv), cp_cell(f.z, hinv), mask);
    const unsigned long long old = atomicExch(head + b, ((unsigned long long)epoch << 32) | (unsigned)d);
    next[d] = (unsigned)(old >> 32) == epoch ? (int)(unsigned)old : -1;
}

// FP64 pair term of the ion-ion sum in scaled units for d = s_j - s_i:
// d (1 + s ln2) 2^-s / s^3 with s = |d|
__device__ __forceinline__ void pair_term_f64(double dx, double dy, double dz, double& tx, double& ty, double& tz)
{
    const double s2 = dx * dx + dy * dy + dz * dz;
    const double s = sqrt(s2);
    const double c = (1.0 + s * 0.69314718055994531) * exp2(-s) / (s2 * s);
    tx = c * dx;
    ty = c * dy;
    tz = c * dz;
}

// Close-pair correction of target i, in scaled units: the sum over ions j with
// |s_j - s_i| < sqrt(dc2) of T(d) - T(d~), T the pair term, d the FP64 separation and
// d~ = fpos_j - fpos_i the separation the FP32 kernels used.  The difference is the
// first-order change of T over delta = d - d~ (computed in FP64, exact up to its last
// bits), evaluated in FP32 at d~:
//   T(d) - T(d~) = c delta + (c'(s) / s) (d~ . delta) d~,  c = (1 + s ln2) 2^-s / s^3,
//   c'(s) / s = -2^-s (3 (1 + s ln2) + (s ln2)^2) / s^5,  s = |d~|;
// it is exact up to (|delta| / s)^2 of T, so pairs with |delta| > 1e-4 s (two ions far
// closer than their rounding would allow at that |s|) take the FP64 difference of the two
// terms instead.  The corrections are added in ascending j (the lists' order depends on
// the atomics that built them), so the sum is deterministic.  pos(j, x, y, z) gives the
// FP64 (unscaled) position of ion j.
constexpr int CP_KEEP = 8;

__device__ __forceinline__ void close_pair_term(float4 fi, float4 fj, double ex, double ey, double ez, float3& t)
{
    // delta = d - d~ (FP64, exact difference of the FP32 values)
    const double gx = (double)fj.x - (double)fi.x, gy = (double)fj.y - (double)fi.y, gz = (double)fj.z - (double)fi.z;
    const double dx = ex - gx, dy = ey - gy, dz = ez - gz;
    const double s2 = gx * gx + gy * gy + gz * gz;
    if (dx * dx + dy * dy + dz * dz > 1e-8 * s2) {
        double t0x, t0y, t0z, t1x, t1y, t1z;
        pair_term_f64(ex, ey, ez, t0x, t0y, t0z);
        pair_term_f64(gx, gy, gz, t1x, t1y, t1z);
        t = make_float3((float)(t0x - t1x), (float)(t0y - t1y), (float)(t0z - t1z));
        return;
    }
    constexpr float LN2 = 0.69314718055994531f;
    const float qx = (float)gx, qy = (float)gy, qz = (float)gz;
    const float q2 = fmaf(qx, qx, fmaf(qy, qy, qz * qz));
    const float ri = rsqrt_approx(q2);
    const float sd = q2 * ri;  // s
    const float e = ex2_approx(-sd);
    const float sl = sd * LN2;
    const float ri2 = ri * ri;
    const float c = e * ri2 * ri * (1.f + sl);
    const float cp = -e * (ri2 * ri2 * ri) * fmaf(sl, sl, 3.f * (1.f + sl));
    const float fx = (float)dx, fy = (float)dy, fz = (float)dz;
    const float proj = cp * fmaf(qx, fx, fmaf(qy, fy, qz * fz));
    t = make_float3(fmaf(c, fx, proj * qx), fmaf(c, fy, proj * qy), fmaf(c, fz, proj * qz));
}

// WIDE lists (a divisor of 8) are walked side by side at a time: 8 for latency (a run of a
// few thousand ions, where each walk step is a memory round trip on the step's critical
// path), 1 where registers are scarce (the batched kernel, held to 128 per thread, whose
// pair tasks would otherwise spill).
template <int WIDE = 8, class PosF>
__device__ void close_pair_corr(const unsigned long long* __restrict__ head, const int* __restrict__ next,
                                const float4* __restrict__ fpos, unsigned mask, float hinv, double dc2,
                                unsigned epoch, int n_live, double ls_inv, int i, double xi, double yi, double zi,
                                PosF pos, double& cx, double& cy, double& cz)
{
    static_assert(WIDE >= 1 && 8 % WIDE == 0, "the eight lists split into equal groups");
    const float4 fi = fpos[i];
    // lower corner of the 2 x 2 x 2 cells around the ion: towards the nearer cell face
    const float ux = fi.x * hinv, uy = fi.y * hinv, uz = fi.z * hinv;
    const int c0x = __float2int_rd(ux), c0y = __float2int_rd(uy), c0z = __float2int_rd(uz);
    const int lx = c0x - (ux - (float)c0x < 0.5f), ly = c0y - (uy - (float)c0y < 0.5f),
              lz = c0z - (uz - (float)c0z < 0.5f);
    const float dc2_f = (float)(1.01 * dc2);
    // the eight bucket words are loaded at once (one memory round trip, not eight)
    unsigned long long hws[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) hws[c] = head[cp_bucket(lx + (c & 1), ly + ((c >> 1) & 1), lz + (c >> 2), mask)];
    cx = cy = cz = 0.0;
    int last = -1;  // with more than CP_KEEP candidates: the pairs up to j = last are summed
    for (int round = 0; round < n_live; ++round) {
        // WIDE lists at a time are walked side by side: each step loads the next entry
        // (position and link) of every one of them at once, so a walk costs one memory round
        // trip per list level, not one per entry.  Candidates: another ion of the same cell,
        // j > last, within the correction distance by the FP32 pre-test (a 1% margin in d^2
        // covers its rounding); the CP_KEEP smallest j are kept.
        int cand[CP_KEEP];
        int nc = 0, over = 0;
#pragma unroll
        for (int g = 0; g < 8; g += WIDE) {
            int jc[WIDE];
#pragma unroll
            for (int w = 0; w < WIDE; ++w) {
                const unsigned long long hw = hws[g + w];
                jc[w] = (unsigned)(hw >> 32) == epoch ? (int)(unsigned)hw : -1;
            }
            for (int level = 0; level < n_live; ++level) {
                float4 fj[WIDE];
                int nx[WIDE];
                bool any = false;
#pragma unroll
                for (int w = 0; w < WIDE; ++w) {
                    nx[w] = -1;
                    if (jc[w] >= 0 && jc[w] < n_live) {
                        fj[w] = fpos[jc[w]];
                        nx[w] = next[jc[w]];
                        any = true;
                    }
                }
                if (!any) break;
#pragma unroll
                for (int w = 0; w < WIDE; ++w) {
                    const int j = jc[w], c = g + w;
                    jc[w] = nx[w];
                    if (!(j >= 0 && j < n_live) || j == i || j <= last) continue;
                    if (cp_cell(fj[w].x, hinv) != lx + (c & 1) || cp_cell(fj[w].y, hinv) != ly + ((c >> 1) & 1) ||
                        cp_cell(fj[w].z, hinv) != lz + (c >> 2))
                        continue;  // another cell sharing the bucket
                    const float gx = fj[w].x - fi.x, gy = fj[w].y - fi.y, gz = fj[w].z - fi.z;
                    if (fmaf(gx, gx, fmaf(gy, gy, gz * gz)) > dc2_f) continue;
                    if (nc < CP_KEEP) {
                        cand[nc++] = j;
                    } else {
                        // keep the CP_KEEP smallest j; the rest wait for the next round
                        over = 1;
                        int m = 0;
                        for (int k = 1; k < CP_KEEP; ++k) m = cand[k] > cand[m] ? k : m;
                        if (j < cand[m]) cand[m] = j;
                    }
                }
            }
        }
        // this round's candidates in ascending j: the FP64 distance test, then the term
        for (int a = 0; a < nc; ++a) {
            int m = a;
            for (int k = a + 1; k < nc; ++k) m = cand[k] < cand[m] ? k : m;
            const int j = cand[m];
            cand[m] = cand[a];
            cand[a] = j;
            double xj, yj, zj;
            pos(j, xj, yj, zj);
            const double ex = (xj - xi) * ls_inv, ey = (yj - yi) * ls_inv, ez = (zj - zi) * ls_inv;
            if (!(ex * ex + ey * ey + ez * ez < dc2)) continue;
            float3 t;
            close_pair_term(fi, fpos[j], ex, ey, ez, t);
            cx += (double)t.x;
            cy += (double)t.y;
            cz += (double)t.z;
        }
        if (!over) break;
        last = cand[nc - 1];
    }
}


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
    // this build of the close-pair lists takes the epoch after the last published one; the
    // last tile publishes it when every tile has entered its ions
    const unsigned cp_ep = cp_next_epoch(*(volatile unsigned*)&C->cp_epoch);
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
            const float4 f = scaled(P, x, y, z, ls_inv);
            B.fpos[d] = f;
            if (P.cp_on) cp_insert(B.cp_head, B.cp_next, P.cp_mask, P.cp_hinv, cp_ep, d, f);
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
                injection_for(P, B, C, C->next_id, r, sn, in);
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
            injection_for(P, B, C, C->next_id, r, sn, in);
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
        const float4 f = scaled(P, ix, iy, iz, ls_inv);
        B.fpos[d] = f;
        if (P.cp_on) cp_insert(B.cp_head, B.cp_next, P.cp_mask, P.cp_hinv, cp_ep, d, f);
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
        C->cp_epoch = cp_ep;
        C->ahead_req_sn = (long long)sn + 1;
        // the next step's injections: the flux rule's Poisson mean plus six deviations, or
        // (one per removed ion) twice this step's removals; the scan draws any beyond
        C->ahead_want = flux ? P.inj_ahead_flux : min(2 * m + 32, INJ_AHEAD);
    }
}

}  // namespace od

#include "od_pairs.cuh"

namespace od {

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
template <int BT, int CP_WIDE = 8>
__device__ __forceinline__ void kick_body(const Phys& P, const Bufs& B, const ForceArgs& F, int mode, int blk)
{
    __shared__ double s_red[BT / 32][3];
    __shared__ double s_Q[MAXD];
    Ctrl* C = B.ctrl;
    const long long step = C->step;
    const int buf = mode == 0 ? (int)((step + 1) & 1) : (int)(step & 1);
    const uint32_t sn = (uint32_t)(step + 1);
    const int i = blk * BT + threadIdx.x;
    const bool live = i < C->n_cur;
    const long long cap = B.cap;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool sym_sums = F.sym && !(P.flags & OD_F_NO_IONION);
    // every load that does not depend on another is issued first (one memory round trip):
    // position, velocity, id, the fixed-point pair sums, the grain charges
    double x = 0, y = 0, z = 0, vx = 0, vy = 0, vz = 0;
    unsigned long long id = 0;
    long long qa = 0, qb = 0, qc = 0;
    long long* A = nullptr;
    if (live) {
        const double* X = B.x[buf];
        x = X[i];
        y = X[cap + i];
        z = X[2 * cap + i];
        if (mode == 0) {
            const double* V = B.v[buf];
            vx = V[i];
            vy = V[cap + i];
            vz = V[2 * cap + i];
            id = B.id[buf][i];
        }
        if (sym_sums) {
            // symmetric kernels (all pairs or the cutoff's listed tile pairs): the fixed-point
            // sum at the ion's position in the pair kernel's order (cleared below)
            A = F.psum + (F.cut ? F.rank[i] : i);
            qa = A[0];
            qb = A[F.psum_ld];
            qc = A[2 * F.psum_ld];
        }
    }
    if ((int)threadIdx.x < P.D) s_Q[threadIdx.x] = C->Q[threadIdx.x];
    __syncthreads();
    int coll = 0;
    if (live) {
        float ax = 0.f, ay = 0.f, az = 0.f;
        if (!(P.flags & OD_F_NO_IONION)) {
            double px = 0.0, py = 0.0, pz = 0.0;  // pair sum in scaled units
            if (F.sym) {
                A[0] = 0;
                A[F.psum_ld] = 0;
                A[2 * F.psum_ld] = 0;
                px = (double)qa * P.qinv;
                py = (double)qb * P.qinv;
                pz = (double)qc * P.qinv;
            } else {
                // ordered-pair kernel: the slots of the blocks that covered this ion's tile,
                // summed in blocks of 16 (all loads of a block issued at once)
                const int t = i / F.TI;
                const long long u0 = (long long)t * F.JS;
                const int ns = (P.flags & OD_F_FP64_PAIRS) ? 1
                                                            : owner_of(u0 + F.JS - 1, F.U, F.G) - owner_of(u0, F.U, F.G) + 1;
                const float4* ps = B.part + i;
                const long long ld = F.n_pad;
                float sx = 0.f, sy = 0.f, sz = 0.f;
                for (int s0 = 0; s0 < ns; s0 += 16) {
                    float bx = 0.f, by = 0.f, bz = 0.f;
                    if (s0 + 16 <= ns) {
                        float4 p[16];
#pragma unroll
                        for (int s = 0; s < 16; ++s) p[s] = __ldcs(ps + (long long)(s0 + s) * ld);
#pragma unroll
                        for (int s = 0; s < 16; ++s) {
                            bx += p[s].x;
                            by += p[s].y;
                            bz += p[s].z;
                        }
                    } else {
                        for (int s = s0; s < ns; ++s) {
                            const float4 p = __ldcs(ps + (long long)s * ld);
                            bx += p.x;
                            by += p.y;
                            bz += p.z;
                        }
                    }
                    sx += bx;
                    sy += by;
                    sz += bz;
                }
                px = sx;
                py = sy;
                pz = sz;
            }
            if (P.cp_on) {
                const double* Xb = B.x[buf];
                double cx, cy, cz;
                close_pair_corr<CP_WIDE>(B.cp_head, B.cp_next, B.fpos, P.cp_mask, P.cp_hinv, P.cp_dc2, C->cp_epoch,
                                         C->n_cur, P.ls_inv, i, x, y, z,
                                         [&](int j, double& xj, double& yj, double& zj) {
                                             xj = Xb[j];
                                             yj = Xb[cap + j];
                                             zj = Xb[2 * cap + j];
                                         },
                                         cx, cy, cz);
                px += cx;
                py += cy;
                pz += cz;
            }
            const double kk = -(double)P.k_ii;
            ax = (float)(px * kk);
            ay = (float)(py * kk);
            az = (float)(pz * kk);
        }
        // bare Coulomb force of the grains (asymmetric model): FP32 terms from FP64
        // separations, like the pair forces
        for (int k = 0; k < P.D; ++k) {
            const float dx = (float)(x - P.gx[k]), dy = (float)(y - P.gy[k]), dz = (float)(z - P.gz[k]);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float ri = rsqrt_approx(r2);
            const float c = (float)(P.kdi * s_Q[k]) * (ri * ri * ri);
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
            const double h = 0.5 * P.dt;
            vx += h * (double)a.x;
            vy += h * (double)a.y;
            vz += h * (double)a.z;
            // Andersen collision with the neutrals: integer threshold on a Philox word
            const uint4 w = philox(P, id, sn, ST_COLL);
            if ((unsigned long long)w.x < P.Tcoll) {
                if (mode == 0 && B.coll_v) {
                    // drawn beside the pair forces (same stream of random numbers)
                    vx = __ldcg(B.coll_v + i);
                    vy = __ldcg(B.coll_v + cap + i);
                    vz = __ldcg(B.coll_v + 2 * cap + i);
                } else {
                    collision_velocity(P, id, sn, vx, vy, vz);
                }
                coll = 1;
            }
            if (P.flags & OD_F_FP32_STATE) vx = rnd32(vx), vy = rnd32(vy), vz = rnd32(vz);
            V[i] = vx;
            V[cap + i] = vy;
            V[2 * cap + i] = vz;
        }
    }
    if (F.sym && !(P.flags & OD_F_NO_IONION)) {
        // the accumulators after the live ions (far-away dummies and padding, whose mutual
        // terms are not zero) are cleared too
        const long long nthr = (long long)((P.N + BT - 1) / BT) * BT;
        for (long long e = C->n_cur + (long long)i; e < F.n_pad; e += nthr) {
            F.psum[e] = 0;
            F.psum[F.psum_ld + e] = 0;
            F.psum[2 * F.psum_ld + e] = 0;
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

// HOIST_WSUM: the grains' window sums are loaded with the other control values (one memory
// round trip fewer in a small run's step); the batched kernel, held to 128 registers, reads
// them where they are added instead
template <bool HOIST_WSUM = true>
__device__ __forceinline__ void dust_body(const Phys& P, const Bufs& B, int nb, int mode)
{
    __shared__ double s_S[MAXD][3];
    __shared__ double s_pm[MAXD][3];
    __shared__ double s_rec[MAXD][REC];
    __shared__ double s_Qd[MAXD];
    Ctrl* C = B.ctrl;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    const int k = threadIdx.x, j = threadIdx.x;
    // the control block's values this tail needs are loaded first, together (one memory
    // round trip): step, removal count, series pointers, each grain's charge, event count
    // and window sums, each event counter
    const long long step = C->step;
    const long long scap = C->series_cap;
    const int m_removed = mode == 0 ? C->removed_total : 0;
    double* const series = C->series;
    int* const evseries = C->evseries;
    double Qk = 0.0, wk[REC], egx = 0.0, egy = 0.0, egz = 0.0;
    int evk = 0;
    if (k < P.D) {
        Qk = C->Q[k];
        evk = C->ev_step[k];
        egx = C->eg[k][0];
        egy = C->eg[k][1];
        egz = C->eg[k][2];
        if (HOIST_WSUM && mode == 0)
#pragma unroll
            for (int t = 0; t < REC; ++t) wk[t] = C->wsum[k][t];
    }
    int evj = 0;
    long long cntj = 0;
    if (mode == 0 && j < EV) {
        evj = C->ev_step[j];
        cntj = C->counters[j];
    }
    // deterministic reduction of the kick's per-block grain sums: warp w of the nw in the
    // CTA takes components w, w + nw, ...; lanes stride the blocks, then a fixed shuffle
    // tree (the same order for any nw)
    for (int pc = warp; pc < P.D * 3; pc += nw) {
        const int kk = pc / 3, c = pc % 3;
        double sum = 0.0;
        for (int b = lane; b < nb; b += 32) sum += B.dpart[((long long)b * MAXD + kk) * 3 + c];
        sum = warp_sum(sum);
        if (lane == 0) s_S[kk][c] = sum;
    }
    // Eq. 3: momentum of the ions each grain absorbed this step (the removed-ion records in
    // rank order: lanes stride them, then the fixed shuffle tree; the first 32 records are
    // loaded beside the count, which is read in the same round trip)
    Rem rm0 = {0.0, 0.0, 0.0, -2, 0};
    if (lane < B.cap) rm0 = B.rem[lane];
    for (int kk = warp; kk < P.D; kk += nw) {
        double px = 0.0, py = 0.0, pz = 0.0;
        for (int r = lane; r < m_removed; r += 32) {
            const Rem rm = r == lane ? rm0 : B.rem[r];
            if (rm.cls == kk) {
                px += rm.vx;
                py += rm.vy;
                pz += rm.vz;
            }
        }
        px = warp_sum(px);
        py = warp_sum(py);
        pz = warp_sum(pz);
        if (lane == 0) {
            s_pm[kk][0] = P.m * px;
            s_pm[kk][1] = P.m * py;
            s_pm[kk][2] = P.m * pz;
        }
    }
    if (k < P.D) s_Qd[k] = Qk;
    __syncthreads();
    if (k < P.D) {
        const double Q = Qk;
        const double ex = egx, ey = egy, ez = egz;
        const double c = P.korb * Q;
        const double fo[3] = {c * s_S[k][0] + ex * Q, c * s_S[k][1] + ey * Q, c * s_S[k][2] + ez * Q};
        for (int t = 0; t < 3; ++t) C->f_orbit[k][t] = fo[t];
        if (mode == 0) {
            // Eq. 2: Coulomb force of the other grains
            double fdd[3] = {0.0, 0.0, 0.0};
            for (int p = 0; p < P.D; ++p) {
                if (p == k) continue;
                const double dx = P.gx[k] - P.gx[p], dy = P.gy[k] - P.gy[p], dz = P.gz[k] - P.gz[p];
                const double d = sqrt(dx * dx + dy * dy + dz * dz);
                const double cc = P.inv4pieps0 * Q * s_Qd[p] / (d * d * d);
                fdd[0] += cc * dx;
                fdd[1] += cc * dy;
                fdd[2] += cc * dz;
            }
            for (int t = 0; t < 3; ++t) {
                s_rec[k][1 + t] = fo[t];
                s_rec[k][4 + t] = fdd[t];
                s_rec[k][7 + t] = s_pm[k][t] / P.dt;
            }
            s_rec[k][10] = 0.0;
            s_rec[k][11] = 0.0;
            s_rec[k][12] = Q * P.E;  // Eq. 4
            // the charge update (explicit: the forces above used the charge before it)
            double Qn = Q;
            if (P.charge_model == OD_Q_CONSISTENT) {
                // absorbed superions plus the OML electron flux at the isolated-sphere potential
                const double a = P.ga[k];
                const double xe = Q * P.inv4pieps0 / a * P.e_over_kTe;
                const double fac = xe <= 0.0 ? exp(xe) : 1.0 + xe;
                const double flux = 4.0 * 3.141592653589793 * a * a * P.Ie0 * fac;
                Qn = Q + P.q * (double)evk - 1.602176634e-19 * flux * P.dt;
                C->Q[k] = Qn;
            }
            s_rec[k][0] = Qn;
            if (step < scap) {
                double* o = series + (step * MAXD + k) * REC;
                for (int t = 0; t < REC; ++t) o[t] = s_rec[k][t];
            }
            if (step + 1 >= P.avg_start)
                for (int t = 0; t < REC; ++t) C->wsum[k][t] = (HOIST_WSUM ? wk[t] : C->wsum[k][t]) + s_rec[k][t];
        }
    }
    if (mode != 0) return;
    // one thread per event counter: record, accumulate, reset for the next step (the grain
    // threads above read their own counts before this block reaches here: the barrier)
    __syncthreads();
    const long long sn = step + 1;
    if (j < EV) {
        if (step < scap) evseries[step * EV + j] = evj;
        C->counters[j] = cntj + evj;
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
