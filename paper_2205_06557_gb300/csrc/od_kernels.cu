// CUDA kernels of the ion-flow-around-dust step for GB300 (sm_103a).
//
// One time step is four kernels, in the canonical order of the method (Sec. 2):
//   k_push_scan  first half kick + drift (velocity Verlet), absorption / outflow test,
//                single-pass decoupled-look-back scan of the removal flags, stable
//                compaction into the other state buffer, and 1:1 re-injection (App. B)
//   k_forces     all-pairs Yukawa ion-ion forces in FP32 (persistent, balanced tiles)
//   k_kick       grain Coulomb force, E_out (App. A) and E_ext on ions, second half kick,
//                Andersen collisions, and the grain-side Yukawa sums of Eq. 1 (FP64); its
//                last block runs the grain tail: Eq. 1-4 terms, charge update, records,
//                time averages
// Every kernel reads the step number from device memory, so a captured graph of one
// step replays without the host.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "od_device.cuh"

namespace od {

// ------------------------------------------------------------ initial fill
__global__ void k_init_ions(Phys P, Bufs B, double ls_inv)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const long long cap = B.cap;
    const unsigned long long id = (unsigned long long)i;
    double x = 0, y = 0, z = 0;
    bool ok = false;
    for (uint32_t att = 0; att < 4096 && !ok; ++att) {
        const uint4 w = philox(P, id, att, ST_INIT_POS);
        const double rho = P.R * sqrt(unif(w.x));
        double s, c;
        sincos(6.283185307179586 * unif(w.y), &s, &c);
        x = rho * c;
        y = rho * s;
        z = P.H * (unif(w.z) - 0.5);
        ok = true;
        for (int k = 0; k < P.D; ++k) {
            const double dx = x - P.gx[k], dy = y - P.gy[k], dz = z - P.gz[k];
            const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            if (d2 <= P.ga2[k]) ok = false;
        }
    }
    if (!ok) atomicOr(&B.ctrl->err, ERR_PLACE);
    const uint4 w = philox(P, id, 0, ST_INIT_VEL);
    double n0, n1, n2, n3;
    box_muller(w.x, w.y, n0, n1);
    box_muller(w.z, w.w, n2, n3);
    double vx = P.sig * n0, vy = P.sig * n1, vz = P.u + P.sig * n2;
    if (P.flags & OD_F_FP32_STATE) {
        x = rnd32(x), y = rnd32(y), z = rnd32(z), vx = rnd32(vx), vy = rnd32(vy), vz = rnd32(vz);
    }
    double* X = B.x[0];
    double* V = B.v[0];
    X[i] = x;
    X[cap + i] = y;
    X[2 * cap + i] = z;
    V[i] = vx;
    V[cap + i] = vy;
    V[2 * cap + i] = vz;
    B.id[0][i] = id;
    B.fpos[i] = scaled(P, x, y, z, ls_inv);
}

// The next step's first injection samples (ids next_id + r, r < ahead_want <= INJ_AHEAD,
// for step ahead_req_sn, all set by this step's scan), launched on a second stream beside
// the pair forces; the next scan uses them where the tag matches and draws the rest
// itself.  The tag is written after the samples.
constexpr int INJ_BT = 32;  // one warp per block: FP64 is slow on this GPU, so the draws
                            // are spread over as many SMs as there are warps of them

__global__ void __launch_bounds__(INJ_BT) k_inject_ahead(Phys P, Bufs B)
{
    __shared__ int s_last;
    Ctrl* C = B.ctrl;
    const long long sn = C->ahead_req_sn;
    const unsigned long long base = C->next_id;
    const int want = min(C->ahead_want, (int)(gridDim.x * INJ_BT));
    const int r = blockIdx.x * INJ_BT + threadIdx.x;
    if (sn > 0 && r < want) {
        Inj o;
        sample_injection(P, base + (unsigned long long)r, (uint32_t)sn, o);
        o.pad = 0;
        B.inj_ahead[r] = o;
    }
    // the last block to finish tags the samples (after every block's have been written)
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&C->inj_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    C->inj_done = 0u;
    if (sn > 0) {
        C->ahead_n = want;
        C->ahead_base = base;
        C->ahead_sn = sn;
    }
}

// This step's collision velocities, beside the pair forces: the ions' order and ids are
// final after the scan, and a collision depends only on (seed, id, step), so the kick
// finds the FP64 Box-Muller draws of its colliding ions ready.
__global__ void k_collide_ahead(Phys P, Bufs B)
{
    const Ctrl* C = B.ctrl;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C->n_cur) return;
    const long long step = C->step;
    const int buf = (int)((step + 1) & 1);
    const uint32_t sn = (uint32_t)(step + 1);
    const unsigned long long id = B.id[buf][i];
    const uint4 w = philox(P, id, sn, ST_COLL);
    if ((unsigned long long)w.x >= P.Tcoll) return;
    double vx, vy, vz;
    collision_velocity(P, id, sn, vx, vy, vz);
    B.coll_v[i] = vx;
    B.coll_v[B.cap + i] = vy;
    B.coll_v[2 * B.cap + i] = vz;
}

int launch_collide_ahead(const Phys& P, const Bufs& B, cudaStream_t s)
{
    if (P.N == 0 || !B.coll_v) return 0;
    k_collide_ahead<<<(P.N + 255) / 256, 256, 0, s>>>(P, B);
    return (int)cudaGetLastError();
}

int launch_inject_ahead(const Phys& P, const Bufs& B, cudaStream_t s)
{
    if (P.N == 0) return 0;
    k_inject_ahead<<<INJ_AHEAD / INJ_BT, INJ_BT, 0, s>>>(P, B);
    return (int)cudaGetLastError();
}

__global__ void k_grain_eout(Phys P, Ctrl* C)
{
    const int k = threadIdx.x;
    if (k >= P.D) return;
    double ex = 0.0, ey = 0.0, ez = 0.0;
    if (P.eout) eout_field(P, P.gx[k], P.gy[k], P.gz[k], ex, ey, ez);
    C->eg[k][0] = ex;
    C->eg[k][1] = ey;
    C->eg[k][2] = ez;
}

int launch_grain_eout(const Phys& P, const Bufs& B, cudaStream_t s)
{
    k_grain_eout<<<1, MAXD, 0, s>>>(P, B.ctrl);
    return (int)cudaGetLastError();
}

// publishes the close-pair lists built by k_fpos (their epoch becomes the current one)
__global__ void k_cp_bump(Ctrl* C) { C->cp_epoch = cp_next_epoch(C->cp_epoch); }

// scaled positions for the pair kernel from state buffer `buf` (entered into the
// close-pair cell lists); dummies beyond N
__global__ void k_fpos(Phys P, Bufs B, int buf, double ls_inv)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n_pad) return;
    const int n = B.ctrl->n_cur;  // ions alive
    if (i < n) {
        const double* X = B.x[buf];
        const float4 f = scaled(P, X[i], X[B.cap + i], X[2 * B.cap + i], ls_inv);
        B.fpos[i] = f;
        if (P.cp_on) cp_insert(B.cp_head, B.cp_next, P.cp_mask, P.cp_hinv, cp_next_epoch(B.ctrl->cp_epoch), i, f);
    } else {
        // far-away dummies: 2^-s underflows to zero, so they add nothing
        const float far = 3.0e4f + 7.0f * (float)(i - n);
        B.fpos[i] = make_float4(far, far, far, 0.0f);
    }
}

// ------------------------------------------------------- single-run kernels
template <int BT>
__global__ void __launch_bounds__(BT) k_push_scan(Phys P, Bufs B, int n_tiles, double ls_inv)
{
    push_scan_body<BT>(P, B, n_tiles, ls_inv, -1);
}

// The kick, then the grain tail in the last block to finish (the grain update reads every
// block's sums; one launch fewer per step than a separate tail kernel)
template <int BT>
__global__ void __launch_bounds__(BT) k_kick(Phys P, Bufs B, ForceArgs F, int mode)
{
    __shared__ int s_last;
    kick_body<BT>(P, B, F, mode, blockIdx.x);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&B.ctrl->kick_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x == 0) B.ctrl->kick_done = 0u;
    dust_body(P, B, (int)gridDim.x, mode);
}


__global__ void k_stats(Phys P, Bufs B, double* out)
{
    const Ctrl* C = B.ctrl;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P.D * REC) return;
    const int k = e / REC, j = e % REC;
    const long long first = P.avg_start > 1 ? P.avg_start : 1;
    const long long cnt = C->step - first + 1;
    double mean = C->wcount > 0 ? C->wsum[k][j] / (double)C->wcount : __longlong_as_double(0x7ff8000000000000ll);
    double se = __longlong_as_double(0x7ff8000000000000ll);
    const long long bl = cnt / 20;
    if (bl >= 1 && C->step <= C->series_cap) {
        double bm[20], mu = 0.0;
        for (int b = 0; b < 20; ++b) {
            double s = 0.0;
            for (long long t = 0; t < bl; ++t) s += C->series[((first - 1 + b * bl + t) * MAXD + k) * REC + j];
            bm[b] = s / (double)bl;
            mu += bm[b] / 20.0;
        }
        double var = 0.0;
        for (int b = 0; b < 20; ++b) var += (bm[b] - mu) * (bm[b] - mu);
        se = sqrt(var / 19.0 / 20.0);
    }
    out[e] = mean;
    out[MAXD * REC + e] = se;
}

// ------------------------------------------------ App. A cavity-potential grid
// I(r0, z0) = int_cyl exp(-|r - r'|/lambda) / |r - r'| d^3r' at each grid node, by slices
// of the cylinder at height z' = z0 + t: in the plane of a slice, polar coordinates about
// the node's projection give the in-plane radial integral in closed form,
//   int_0^S s exp(-sqrt(s^2 + t^2)/lambda) / sqrt(s^2 + t^2) ds
//       = lambda (exp(-|t|/lambda) - exp(-sqrt(S^2 + t^2)/lambda)),
// S(psi) = -r0 cos psi + sqrt(R^2 - r0^2 sin^2 psi) the distance to the slice's rim in
// direction psi.  The first term integrates in closed form over psi and t:
// 2 pi lambda^2 (2 - exp(-a/lambda) - exp(-b/lambda)), a and b the distances from the
// node to the end faces.  The second is smooth in psi (twice the integral over [0, pi])
// and in t on each side of the node (t in [0, a] and [0, b]); both go to Gauss-Legendre.
// On the rim (r0 = R) S vanishes for psi < pi/2, where that part is exp(-|t|/lambda)
// again and integrates in closed form.
__global__ void k_eout_grid(double R, double H, double lam, int nx, int nz, int nq, const double* __restrict__ glx,
                            const double* __restrict__ glw, double* __restrict__ out)
{
    __shared__ double s_part[128];
    const int node = blockIdx.x;
    const int kr = node / (nz + 1), kz = node % (nz + 1);
    const double r0 = R * kr / nx, z0 = 0.5 * H * kz / nz;
    const double a = 0.5 * H - z0, b = 0.5 * H + z0;
    const double PI = 3.141592653589793;
    const bool rim = kr == nx;
    const double p0 = rim ? 0.5 * PI : 0.0, p1 = PI;  // the psi range with S > 0
    double acc = 0.0;
    // one (psi node, side of the node) pair per thread
    for (int w = threadIdx.x; w < 2 * nq; w += blockDim.x) {
        const int iq = w >> 1, side = w & 1;
        const double L = side == 0 ? a : b;
        if (!(L > 0.0)) continue;
        const double psi = 0.5 * (p0 + p1) + 0.5 * (p1 - p0) * glx[iq];
        const double wpsi = 0.5 * (p1 - p0) * glw[iq];
        double sp, cp;
        sincos(psi, &sp, &cp);
        const double S = rim ? -2.0 * R * cp : -r0 * cp + sqrt(fmax(R * R - r0 * r0 * sp * sp, 0.0));
        const double S2 = S * S;
        double sum = 0.0;
        for (int it = 0; it < nq; ++it) {
            const double t = 0.5 * L * (1.0 + glx[it]);
            sum += glw[it] * exp(-sqrt(S2 + t * t) / lam);
        }
        acc += wpsi * 0.5 * L * sum;
    }
    s_part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s_part[threadIdx.x] += s_part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double ea = exp(-a / lam), eb = exp(-b / lam);
        double I = 2.0 * PI * lam * lam * (2.0 - ea - eb) - 2.0 * lam * s_part[0];
        // rim: psi in [0, pi/2] (S = 0), both signs of psi
        if (rim) I -= 2.0 * (0.5 * PI) * lam * lam * ((1.0 - ea) + (1.0 - eb));
        out[node] = I;
    }
}

// ------------------------------------------------ OML floating charge (Sec. 2 "oml")
// One CTA per grain.  The floating potential phi <= 0 balances the OML ion current of a
// drifting Maxwellian (thermal speed sig, drift u; cross-section pi a^2 (1 - 2 Z e phi /
// (m v^2))) against the Boltzmann electron current
//   I_e = e Z n pi a^2 sqrt(8 k T_e / (pi m_e)) exp(e phi / k T_e);
// the ion current is one speed integral of v^3 sigma(v) times the angular average of the
// shifted Maxwellian, Gauss-Legendre on [0, u] and [u, u + 14 sig] (the nodes split over
// the CTA, summed in a fixed order).  Bisection on [-200 k T_e / e, 0] to 1e-14 k T_e / e;
// Q = 4 pi eps0 a phi.
constexpr int OML_BT = 256;

struct OmlArgs {
    double n, m, sig, u, Z, kTe_over_e, Ie_coef;  // Ie_coef = e Z n sqrt(8 k T_e / (pi m_e)) pi
    int D;
    double a[MAXD];
};

__device__ double oml_block_sum(double v, double* s_w)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) s_w[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int k = 0; k < OML_BT / 32; ++k) t += s_w[k];
    return t;
}

__global__ void __launch_bounds__(OML_BT) k_oml_charge(OmlArgs A, int nq, const double* __restrict__ glx,
                                                     const double* __restrict__ glw, Ctrl* C)
{
    __shared__ double s_w[OML_BT / 32];
    const int k = blockIdx.x;
    const double a = A.a[k], PI = 3.141592653589793, QE = 1.602176634e-19, EPS0 = 8.8541878128e-12;
    const double s2 = A.sig * A.sig;
    const int nseg = A.u > 0.0 ? 2 : 1;
    const double e0 = 0.0, e1 = A.u > 0.0 ? A.u : 0.0, e2 = e1 + 14.0 * A.sig;
    const double norm = A.Z * QE * A.n * pow(2.0 * PI * s2, -1.5);
    double lo = -200.0 * A.kTe_over_e, hi = 0.0;
    for (int it = 0; it < 200 && hi - lo > 1e-14 * A.kTe_over_e; ++it) {
        const double phi = 0.5 * (lo + hi);
        double part = 0.0;
        for (int q = threadIdx.x; q < nseg * nq; q += OML_BT) {
            const int seg = q / nq, iq = q % nq;
            const double pa = seg == 0 ? (nseg == 2 ? e0 : e0) : e1, pb = seg == 0 ? (nseg == 2 ? e1 : e2) : e2;
            const double v = 0.5 * (pa + pb) + 0.5 * (pb - pa) * glx[iq];
            const double wv = 0.5 * (pb - pa) * glw[iq];
            if (!(v > 0.0)) continue;
            const double cross = PI * a * a * (1.0 - 2.0 * A.Z * QE * phi / (A.m * v * v));
            double ang;
            if (A.u <= 0.0) {
                ang = 4.0 * PI * exp(-v * v / (2.0 * s2));
            } else {
                const double x = v * A.u / s2;
                ang = 2.0 * PI * (exp(-(v - A.u) * (v - A.u) / (2.0 * s2)) - exp(-(v + A.u) * (v + A.u) / (2.0 * s2))) / x;
            }
            part += wv * v * v * v * cross * ang;
        }
        const double Ii = norm * oml_block_sum(part, s_w);
        const double Ie = A.Ie_coef * a * a * exp(phi / A.kTe_over_e);
        if (Ii - Ie > 0.0) lo = phi;
        else hi = phi;
    }
    if (threadIdx.x == 0) C->Q[k] = 4.0 * PI * EPS0 * a * 0.5 * (lo + hi);
}

int launch_oml_charge(const Phys& P, const Bufs& B, double n_inf, double m_i, double Z, double T_e, int nq,
                      const double* glx, const double* glw, cudaStream_t s)
{
    if (P.D == 0) return 0;
    OmlArgs A{};
    const double KB = 1.380649e-23, QE = 1.602176634e-19, ME = 9.1093837015e-31, PI = 3.141592653589793;
    A.n = n_inf;
    A.m = m_i;
    A.sig = P.sig;
    A.u = P.u;
    A.Z = Z;
    A.kTe_over_e = KB * T_e / QE;
    A.Ie_coef = QE * Z * n_inf * sqrt(8.0 * KB * T_e / (PI * ME)) * PI;
    A.D = P.D;
    for (int k = 0; k < P.D; ++k) A.a[k] = P.ga[k];
    k_oml_charge<<<P.D, OML_BT, 0, s>>>(A, nq, glx, glw, B.ctrl);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------- launchers
static int ck(cudaError_t e)
{
    return e == cudaSuccess ? 0 : (int)e;
}

int push_tile() { return PUSH_BT; }
int kick_block() { return KICK_BT; }

int launch_init_ions(const Phys& P, const Bufs& B, cudaStream_t s)
{
    if (P.N == 0) return 0;
    const double ls_inv = 1.4426950408889634 * P.lam_inv;
    k_init_ions<<<(P.N + 255) / 256, 256, 0, s>>>(P, B, ls_inv);
    return ck(cudaGetLastError());
}

int launch_cp_bump(const Bufs& B, cudaStream_t s)
{
    k_cp_bump<<<1, 1, 0, s>>>(B.ctrl);
    return ck(cudaGetLastError());
}

int launch_fpos(const Phys& P, const Bufs& B, int buf, cudaStream_t s)
{
    if (P.n_pad == 0) return 0;
    const double ls_inv = 1.4426950408889634 * P.lam_inv;
    k_fpos<<<(P.n_pad + 255) / 256, 256, 0, s>>>(P, B, buf, ls_inv);
    if (P.cp_on) k_cp_bump<<<1, 1, 0, s>>>(B.ctrl);
    return ck(cudaGetLastError());
}

int launch_pad(const Phys& P, const Bufs& B, cudaStream_t s) { return launch_fpos(P, B, 0, s); }

int launch_push_scan(const Phys& P, const Bufs& B, cudaStream_t s)
{
    if (P.N == 0) return 0;
    const double ls_inv = 1.4426950408889634 * P.lam_inv;
    const int n_tiles = (P.N + PUSH_BT - 1) / PUSH_BT;
    k_push_scan<PUSH_BT><<<n_tiles, PUSH_BT, 0, s>>>(P, B, n_tiles, ls_inv);
    return ck(cudaGetLastError());
}

// pair-kernel variants (threads per block, targets per thread): ordered-pair kernels
// k_forces, symmetric ones k_forces_sym, then symmetric ones on packed FP32 pairs
// k_forces_sym2; targets per tile BT * IPT never exceed 1024, the padding granularity of
// the position buffer
#define OD_FORCE_VARIANTS(X) X(64, 1) X(64, 2) X(128, 2) X(128, 4) X(256, 2) X(256, 4) X(128, 8) X(64, 8)
#define OD_SYM_VARIANTS(X) X(128, 2) X(128, 4) X(256, 2) X(256, 4)
#define OD_SYM2_VARIANTS(X) X(128, 2) X(128, 4) X(256, 2) X(256, 4) X(128, 8) X(64, 8) X(32, 8)

static const ForceVariant kVariants[] = {
#define OD_V(bt, ipt) {bt, ipt, 0},
    OD_FORCE_VARIANTS(OD_V)
#undef OD_V
#define OD_V(bt, ipt) {bt, ipt, 1},
    OD_SYM_VARIANTS(OD_V)
#undef OD_V
#define OD_V(bt, ipt) {bt, ipt, 2},
    OD_SYM2_VARIANTS(OD_V)
#undef OD_V
};

int num_force_variants() { return (int)(sizeof(kVariants) / sizeof(kVariants[0])); }
ForceVariant force_variant(int v) { return kVariants[v]; }

static void* variant_fn(int v)
{
    static void* const fns[] = {
#define OD_V(bt, ipt) (void*)k_forces<bt, ipt>,
        OD_FORCE_VARIANTS(OD_V)
#undef OD_V
#define OD_V(bt, ipt) (void*)k_forces_sym<bt, ipt>,
        OD_SYM_VARIANTS(OD_V)
#undef OD_V
#define OD_V(bt, ipt) (void*)k_forces_sym2<bt, ipt>,
        OD_SYM2_VARIANTS(OD_V)
#undef OD_V
    };
    return fns[v];
}

int force_blocks_per_sm(int v)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, variant_fn(v), kVariants[v].BT, 0) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

// Study-only FP64 pair forces (precision study of the FP32 kernels): one target per
// thread, sources staged through shared memory, everything in FP64 from the FP64 state
// (libm exp2 and sqrt), written as partial slot 0 in the scaled units of the FP32
// kernels: sum_j (1 + s ln2) 2^-s d / s^3 with d = (r_j - r_i) log2(e) / lambda_De.
// after_push: the step's new positions (the push writes them to the other buffer).
constexpr int F64_BT = 128;

__global__ void __launch_bounds__(F64_BT) k_forces_f64(Phys P, Bufs B, int after_push, double ls_inv)
{
    __shared__ double sx[F64_BT], sy[F64_BT], sz[F64_BT];
    const long long step = B.ctrl->step;
    const int buf = after_push ? (int)((step + 1) & 1) : (int)(step & 1);
    const double* X = B.x[buf];
    const int n = B.ctrl->n_cur;
    const long long cap = B.cap;
    const int i = blockIdx.x * F64_BT + threadIdx.x;
    const double xi = i < n ? X[i] * ls_inv : 0.0, yi = i < n ? X[cap + i] * ls_inv : 0.0;
    const double zi = i < n ? X[2 * cap + i] * ls_inv : 0.0;
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int j0 = 0; j0 < n; j0 += F64_BT) {
        __syncthreads();
        const int j = j0 + threadIdx.x;
        sx[threadIdx.x] = j < n ? X[j] * ls_inv : 0.0;
        sy[threadIdx.x] = j < n ? X[cap + j] * ls_inv : 0.0;
        sz[threadIdx.x] = j < n ? X[2 * cap + j] * ls_inv : 0.0;
        __syncthreads();
        const int jn = min(F64_BT, n - j0);
        for (int jj = 0; jj < jn; ++jj) {
            if (j0 + jj == i) continue;
            const double dx = sx[jj] - xi, dy = sy[jj] - yi, dz = sz[jj] - zi;
            const double s2 = dx * dx + dy * dy + dz * dz;
            const double sd = sqrt(s2);
            const double c = (1.0 + sd * 0.69314718055994531) * exp2(-sd) / (s2 * sd);
            ax += c * dx;
            ay += c * dy;
            az += c * dz;
        }
    }
    if (i < n) B.part[i] = make_float4((float)ax, (float)ay, (float)az, 0.f);
}

int launch_forces_f64(const Phys& P, const Bufs& B, int after_push, cudaStream_t s)
{
    if (P.N == 0 || (P.flags & OD_F_NO_IONION)) return 0;
    const double ls_inv = 1.4426950408889634 * P.lam_inv;
    k_forces_f64<<<(P.N + F64_BT - 1) / F64_BT, F64_BT, 0, s>>>(P, B, after_push, ls_inv);
    return ck(cudaGetLastError());
}

int launch_forces(const Phys& P, const Bufs& B, const ForceArgs& F, int v, cudaStream_t s)
{
    if (P.N == 0 || (P.flags & OD_F_NO_IONION) || F.G == 0) return 0;
    if (v < 0 || v >= num_force_variants() || (kVariants[v].sym == 2 && !F.sched)) return (int)cudaErrorInvalidValue;
    int idx = 0;
#define OD_V(bt, ipt)                                                \
    if (v == idx++) {                                                \
        k_forces<bt, ipt><<<F.G, bt, 0, s>>>(B.fpos, B.part, F);     \
        return ck(cudaGetLastError());                               \
    }
    OD_FORCE_VARIANTS(OD_V)
#undef OD_V
#define OD_V(bt, ipt)                                        \
    if (v == idx++) {                                        \
        k_forces_sym<bt, ipt><<<F.G, bt, 0, s>>>(B.fpos, F); \
        return ck(cudaGetLastError());                       \
    }
    OD_SYM_VARIANTS(OD_V)
#undef OD_V
#define OD_V(bt, ipt)                                         \
    if (v == idx++) {                                         \
        k_forces_sym2<bt, ipt><<<F.G, bt, 0, s>>>(B.fpos, F); \
        return ck(cudaGetLastError());                        \
    }
    OD_SYM2_VARIANTS(OD_V)
#undef OD_V
    return (int)cudaErrorInvalidValue;
}

int launch_kick(const Phys& P, const Bufs& B, const ForceArgs& F, int mode, cudaStream_t s)
{
    if (P.N == 0) return 0;
    k_kick<KICK_BT><<<(P.N + KICK_BT - 1) / KICK_BT, KICK_BT, 0, s>>>(P, B, F, mode);
    return ck(cudaGetLastError());
}


// host interface layouts: the ABI's interleaved [n][3] arrays <-> the device's [3][cap]
// structure of arrays (and the float4 accelerations), converted on the device so that a
// host array moves as one contiguous copy
__global__ void k_aos_to_soa(const double* __restrict__ aos, double* __restrict__ soa, int n, long long cap)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    soa[i] = aos[3 * (long long)i];
    soa[cap + i] = aos[3 * (long long)i + 1];
    soa[2 * cap + i] = aos[3 * (long long)i + 2];
}

__global__ void k_soa_to_aos(const double* __restrict__ soa, double* __restrict__ aos, int n, long long cap)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    aos[3 * (long long)i] = soa[i];
    aos[3 * (long long)i + 1] = soa[cap + i];
    aos[3 * (long long)i + 2] = soa[2 * cap + i];
}

__global__ void k_acc_to_aos(const float4* __restrict__ acc, double* __restrict__ aos, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 a = acc[i];
    aos[3 * (long long)i] = a.x;
    aos[3 * (long long)i + 1] = a.y;
    aos[3 * (long long)i + 2] = a.z;
}

__global__ void k_aos_to_acc(const double* __restrict__ aos, float4* __restrict__ acc, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    acc[i] = make_float4((float)aos[3 * (long long)i], (float)aos[3 * (long long)i + 1], (float)aos[3 * (long long)i + 2],
                         0.f);
}

int launch_layout(int kind, const void* src, void* dst, int n, long long cap, cudaStream_t s)
{
    if (n <= 0) return 0;
    const int g = (n + 255) / 256;
    switch (kind) {
    case 0: k_aos_to_soa<<<g, 256, 0, s>>>((const double*)src, (double*)dst, n, cap); break;
    case 1: k_soa_to_aos<<<g, 256, 0, s>>>((const double*)src, (double*)dst, n, cap); break;
    case 2: k_acc_to_aos<<<g, 256, 0, s>>>((const float4*)src, (double*)dst, n); break;
    default: k_aos_to_acc<<<g, 256, 0, s>>>((const double*)src, (float4*)dst, n); break;
    }
    return ck(cudaGetLastError());
}

// n(r, z) binning of the ions at the end of a step (observability): bin indices from
// the FP64 positions with explicitly rounded operations (no contraction), so a host
// binning that evaluates r = sqrt(x*x + y*y), r * (nr / R) and (z + H/2) * (nz / H)
// in IEEE FP64 finds the same bins; integer counts, so the result does not depend on the
// order of the atomics.  Small maps are privatised in shared memory per block.
constexpr int HIST_SMEM_BINS = 12288;

__global__ void k_hist(Phys P, Bufs B, unsigned long long* counts, int nr, int nz, double inv_dr, double inv_dz)
{
    extern __shared__ unsigned s_h[];
    const int nb = nr * nz;
    const bool priv = nb <= HIST_SMEM_BINS;
    if (priv)
        for (int b = threadIdx.x; b < nb; b += blockDim.x) s_h[b] = 0u;
    __syncthreads();
    const long long step = B.ctrl->step;  // positions after step n live in buffer n & 1
    const double* X = B.x[step & 1];
    const double hz = 0.5 * P.H;
    const int n = B.ctrl->n_cur;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double x = X[i], y = X[B.cap + i], z = X[2 * B.cap + i];
        const double r = __dsqrt_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)));
        const int ir = min(max((int)__dmul_rn(r, inv_dr), 0), nr - 1);
        const int iz = min(max((int)__dmul_rn(__dadd_rn(z, hz), inv_dz), 0), nz - 1);
        if (priv) atomicAdd(&s_h[iz * nr + ir], 1u);
        else atomicAdd(&counts[iz * nr + ir], 1ull);
    }
    if (priv) {
        __syncthreads();
        for (int b = threadIdx.x; b < nb; b += blockDim.x)
            if (s_h[b]) atomicAdd(&counts[b], (unsigned long long)s_h[b]);
    }
}

int launch_hist(const Phys& P, const Bufs& B, unsigned long long* counts, int nr, int nz, double inv_dr, double inv_dz,
                int sms, cudaStream_t s)
{
    if (P.N == 0) return 0;
    const int nb = nr * nz;
    const size_t smem = nb <= HIST_SMEM_BINS ? sizeof(unsigned) * nb : 0;
    const int grid = std::max(1, std::min((P.N + 255) / 256, 2 * sms));
    k_hist<<<grid, 256, smem, s>>>(P, B, counts, nr, nz, inv_dr, inv_dz);
    return ck(cudaGetLastError());
}

int launch_stats(const Phys& P, const Bufs& B, double* out, cudaStream_t s)
{
    k_stats<<<1, 128, 0, s>>>(P, B, out);
    return ck(cudaGetLastError());
}

int launch_eout_grid(double R, double H, double lam, int nx, int nz, int nq, const double* glx, const double* glw,
                     double* out, cudaStream_t s)
{
    k_eout_grid<<<(nx + 1) * (nz + 1), 128, 0, s>>>(R, H, lam, nx, nz, nq, glx, glw, out);
    return ck(cudaGetLastError());
}

}  // namespace od

// ---------------------------------------------- no-allocation pair forces
// A variant of the pair-force computation for callers that cannot allocate device
// memory.  Its scratch (scaled positions, the per-chunk partial sums, the close-pair
// cell buckets and links and one bound word) lives in one file-scope device array of
// fixed size that every GPU loading this library holds until the process exits.  Host
// code only sees a stand-in for the array's name, so the device address is looked up
// with cudaGetSymbolAddress (once per device and context) and passed to the kernels.
namespace od {
namespace {
constexpr int kStaticBT = 128, kStaticIPT = 2, kStaticTI = kStaticBT * kStaticIPT;
constexpr int kStaticSlots = 8;                       // source chunks per target tile
constexpr int kStaticBuckets = 2 * OD_STATIC_MAX_IONS; // close-pair cell buckets (u64 each)
// layout in float4 units: positions, partial slots, buckets, links, bound word
constexpr long long kOffPart = OD_STATIC_MAX_IONS;
constexpr long long kOffHead = kOffPart + (long long)OD_STATIC_MAX_IONS * kStaticSlots;
constexpr long long kOffNext = kOffHead + kStaticBuckets / 2;
constexpr long long kOffBound = kOffNext + OD_STATIC_MAX_IONS / 4;
constexpr long long kStaticFloat4 = kOffBound + 1;
static_assert(OD_STATIC_MAX_IONS % kStaticTI == 0, "capacity must be a whole number of tiles");
static_assert((kStaticBuckets & (kStaticBuckets - 1)) == 0, "bucket count must be a power of two");
}  // namespace

static __device__ __align__(256) float4 g_static_scratch[kStaticFloat4];

// correction distance and cell width (scaled units) from the largest |s|: pairs closer
// than 0.005 max(1, |s|max / 4) get their FP64 value (cells 2.1 times as wide)
__device__ __forceinline__ void static_cp_params(const unsigned* bound, double& dc2, float& hinv)
{
    const double smax = (double)__uint_as_float(*bound);
    const double dc = 0.005 * fmax(1.0, 0.25 * smax);
    dc2 = dc * dc;
    hinv = (float)(1.0 / (2.1 * dc));
}

// largest |coordinate| in scaled units (non-negative floats order like their bits)
__global__ void k_static_bound(const double* __restrict__ x, int n, double ls_inv, unsigned* __restrict__ bound)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float m = 0.f;
    if (i < n)
        m = fmaxf(fabsf((float)(x[3 * i] * ls_inv)), fmaxf(fabsf((float)(x[3 * i + 1] * ls_inv)),
                                                         fabsf((float)(x[3 * i + 2] * ls_inv))));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(bound, __float_as_uint(m));
}

// scaled FP32 positions, entered into the close-pair cells; padding beyond n goes
// 256 scaled units (a factor 2^-256 in the pair term: exactly zero in FP32) past the
// largest coordinate and 256 apart
__global__ void k_static_scale(const double* __restrict__ x, int n, int n_pad, double ls_inv, float4* __restrict__ fpos,
                               unsigned long long* __restrict__ head, int* __restrict__ next,
                               const unsigned* __restrict__ bound, unsigned epoch)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    if (i < n) {
        const float4 f = make_float4((float)(x[3 * i] * ls_inv), (float)(x[3 * i + 1] * ls_inv),
                                     (float)(x[3 * i + 2] * ls_inv), 0.0f);
        fpos[i] = f;
        double dc2;
        float hinv;
        static_cp_params(bound, dc2, hinv);
        cp_insert(head, next, (unsigned)kStaticBuckets - 1u, hinv, epoch, i, f);
    } else {
        const float far = __uint_as_float(*bound) + 256.0f * (float)(i - n + 1);
        fpos[i] = make_float4(far, far, far, 0.0f);
    }
}

// sum of each ion's partial slots, plus the close-pair correction, times -k
__global__ void k_static_reduce(const float4* __restrict__ part, const double* __restrict__ x, int n, int n_pad,
                                int slots, double ls_inv, double kscale, const float4* __restrict__ fpos,
                                const unsigned long long* __restrict__ head, const int* __restrict__ next,
                                const unsigned* __restrict__ bound, unsigned epoch, float* __restrict__ a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float ax = 0.f, ay = 0.f, az = 0.f;
    for (int s = 0; s < slots; ++s) {
        const float4 p = part[(long long)s * n_pad + i];
        ax += p.x;
        ay += p.y;
        az += p.z;
    }
    double dc2;
    float hinv;
    static_cp_params(bound, dc2, hinv);
    double cx, cy, cz;
    close_pair_corr(head, next, fpos, (unsigned)kStaticBuckets - 1u, hinv, dc2, epoch, n, ls_inv, i, x[3 * i],
                    x[3 * i + 1], x[3 * i + 2],
                    [&](int j, double& xj, double& yj, double& zj) {
                        xj = x[3 * j];
                        yj = x[3 * j + 1];
                        zj = x[3 * j + 2];
                    },
                    cx, cy, cz);
    a[3 * i] = (float)(-kscale * ((double)ax + cx));
    a[3 * i + 1] = (float)(-kscale * ((double)ay + cy));
    a[3 * i + 2] = (float)(-kscale * ((double)az + cz));
}

// The array's device address in the current context of device dev, and a fresh epoch
// for the close-pair buckets (each call's lists get their own tag).  The address is
// looked up again when the device's context changes (e.g. after cudaDeviceReset, which
// reloads the module): the context is identified through the driver entry point
// cuCtxGetCurrent, fetched from the runtime so that the library needs no link to libcuda.
static float4* static_scratch_address(int dev, int* rc, unsigned* epoch)
{
    static std::mutex mu;
    static float4* addr[256] = {nullptr};
    static void* ctx_of[256] = {nullptr};
    static unsigned ep[256] = {0};
    *rc = OD_OK;
    if (dev < 0 || dev >= 256) {
        *rc = OD_EINVAL;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    typedef int (*CtxGetCurrent)(void**);
    static CtxGetCurrent get_ctx = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_ctx = (CtxGetCurrent)fn;
        cudaGetLastError();
    }
    void* ctx = nullptr;
    if (get_ctx) get_ctx(&ctx);
    if (!addr[dev] || ctx != ctx_of[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            *rc = OD_ECUDA;
            set_global_error(std::string("cudaGetSymbolAddress of the static scratch failed: ") + cudaGetErrorString(e));
            return nullptr;
        }
        addr[dev] = (float4*)p;
        ctx_of[dev] = ctx;
        ep[dev] = 0;  // a new context starts from a zeroed array
    }
    ep[dev] = ep[dev] + 1u == 0u ? 1u : ep[dev] + 1u;
    *epoch = ep[dev];
    return addr[dev];
}

}  // namespace od

extern "C" int od_pair_accel_static(const double* x, int64_t n, double lambda_De, double k, float* a, void* stream)
{
    using namespace od;
    if (n < 0 || n > OD_STATIC_MAX_IONS) {
        set_global_error("od_pair_accel_static: n must be in 0.." + std::to_string(OD_STATIC_MAX_IONS));
        return OD_EINVAL;
    }
    if (!(lambda_De > 0.0) || !std::isfinite(lambda_De) || !std::isfinite(k) || (n > 0 && (!x || !a))) {
        set_global_error("od_pair_accel_static: lambda_De must be finite and > 0, k finite, x and a non-NULL");
        return OD_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        set_global_error("od_pair_accel_static: no current CUDA device");
        return OD_ENODEV;
    }
    int rc = OD_OK;
    unsigned epoch = 0;
    float4* base = static_scratch_address(dev, &rc, &epoch);
    if (!base) return rc;
    if (n == 0) return OD_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const double ls_inv = 1.4426950408889634 / lambda_De;  // log2(e) / lambda_De
    ForceArgs F{};
    F.TI = kStaticTI;
    F.n_pad = (int)((n + kStaticTI - 1) / kStaticTI * kStaticTI);
    const int n_it = F.n_pad / kStaticTI;
    int js = std::min(kStaticSlots, F.n_pad / kStaticBT);
    F.JC = ((F.n_pad + js - 1) / js + kStaticBT - 1) / kStaticBT * kStaticBT;
    F.JS = (F.n_pad + F.JC - 1) / F.JC;
    F.U = (long long)n_it * F.JS;
    F.G = (int)F.U;  // one unit per block: the partial slot of a block is its chunk index
    F.W = F.JS;
    float4* fpos = base;
    float4* part = base + kOffPart;
    unsigned long long* head = (unsigned long long*)(base + kOffHead);
    int* next = (int*)(base + kOffNext);
    unsigned* bound = (unsigned*)(base + kOffBound);
    // the bound word is the one value that must start at zero on every call
    cudaError_t e = cudaMemsetAsync(bound, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) {
        k_static_bound<<<(int)((n + 255) / 256), 256, 0, s>>>(x, (int)n, ls_inv, bound);
        k_static_scale<<<(F.n_pad + 255) / 256, 256, 0, s>>>(x, (int)n, F.n_pad, ls_inv, fpos, head, next, bound, epoch);
        k_forces<kStaticBT, kStaticIPT><<<F.G, kStaticBT, 0, s>>>(fpos, part, F);
        const double kscale = k * ls_inv * ls_inv;
        k_static_reduce<<<(int)((n + 255) / 256), 256, 0, s>>>(part, x, (int)n, F.n_pad, F.JS, ls_inv, kscale, fpos,
                                                               head, next, bound, epoch, a);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_global_error(std::string("od_pair_accel_static: launch failed: ") + cudaGetErrorString(e));
        return OD_ECUDA;
    }
    return OD_OK;
}
