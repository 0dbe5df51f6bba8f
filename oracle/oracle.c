/*
 * Oracle for the ion-flow-around-dust time step (OpenDust, arXiv 2205.06557).
 *
 * TEST INFRASTRUCTURE ONLY: a plain FP64 CPU restatement of the method, used to
 * check the CUDA library.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code with the CUDA library.
 *
 * Everything is written for a reader holding the paper:
 *   - ions are "superions" of w real ions, charge q = w Z e, mass m = w m_i (Sec. 2);
 *   - ion-ion forces are Yukawa-screened with the electron Debye length, ion-dust
 *     forces on ions are bare Coulomb, forces on dust from ions are Yukawa (Sec. 2, Eq. 1);
 *   - ions outside the domain act through the cavity field E_out (App. A);
 *   - ions move by velocity Verlet; collisions replace the velocity with a neutral
 *     Maxwellian sample at a constant frequency (Andersen thermostat, Sec. 2);
 *   - ions that leave or hit a grain are replaced 1:1 on the boundary by the
 *     flux-conserving rule of App. B; absorbed ions charge the grain and transfer
 *     momentum (Eq. 3, Sec. 2 charging models);
 *   - per-step dust records hold q and the four force terms of Eqs. 1-4.
 *
 * Where the paper is silent the readings are documented beside the code and in the
 * design notes: step order, RNG layout (Philox4x32-10 keyed by seed, counter =
 * (ion id, step, stream)), the collision probability 1-exp(-nu dt), integer
 * thresholds for random decisions, the inverse-CDF sampler, the absorption test
 * at the end point of the step, and the continuum reading of App. A's ion sum.
 *
 * The ion-ion loop over target ions may run under OpenMP; each target's sum keeps
 * the same serial order, so results do not depend on the thread count.
 */
#include "oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* CODATA 2018 values */
static const double QE = 1.602176634e-19;    /* C */
static const double KB = 1.380649e-23;       /* J/K */
static const double EPS0 = 8.8541878128e-12; /* F/m */
static const double ME = 9.1093837015e-31;   /* kg */
#define PI 3.14159265358979323846
#define TWO32 4294967296.0

/* Philox streams (fourth counter word) */
enum { ST_INIT_POS = 0, ST_INIT_VEL = 1, ST_COLL = 2, ST_COLL_VEL = 3, ST_INJ_A = 4, ST_INJ_B = 5, ST_INJ_N = 6 };

struct orc_state {
    orc_params p;
    double lam;   /* electron Debye length */
    double cs;    /* ion sound speed sqrt(Z k T_e / m_i) */
    double sig;   /* ion thermal speed sqrt(k T_i / m_i) */
    double sig_n; /* neutral thermal speed sqrt(k T_n / m_i) */
    double u;     /* flow speed */
    double E;     /* driving field along z */
    double q, m;  /* superion charge and mass */
    double pb, pt, ps;
    uint64_t Tb, Tbt, Tcoll;
    double pcoll;
    double alpha[15];
    double Ie0;   /* electron flux per unit area at zero potential, 1/(m^2 s) */
    double inj_rate; /* superions entering through the three faces per second (App. B) */
    int64_t N, next_id, step;
    double *x, *v, *a;
    uint64_t* id;
    double Q[ORC_MAX_DUST];
    int64_t cap;
    double* rec;
    int32_t* ev;
};

/* ------------------------------------------------------------------ Philox */
/* Philox4x32-10, Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
 * 1, 2, 3" (SC'11): ten rounds of two 32x32->64 multiplies, with the key bumped by
 * the Weyl constants between rounds. */
void orc_philox(const uint32_t key[2], const uint32_t ctr[4], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

static void draw(const orc_state* s, uint64_t id, uint32_t word2, uint32_t stream, uint32_t out[4])
{
    uint32_t key[2] = {(uint32_t)s->p.seed, (uint32_t)(s->p.seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), word2, stream};
    orc_philox(key, ctr, out);
}

/* uniform in (0,1), never 0 or 1 */
static double unif(uint32_t w) { return ((double)w + 0.5) / TWO32; }

/* Box-Muller: two independent standard normals from two uniforms */
static void box_muller(uint32_t wa, uint32_t wb, double* n0, double* n1)
{
    double rad = sqrt(-2.0 * log(unif(wa)));
    double t = 2.0 * PI * unif(wb);
    *n0 = rad * cos(t);
    *n1 = rad * sin(t);
}

/* ------------------------------------------------------------- App. B math */
static double ncdf(double z) { return 0.5 * erfc(-z / sqrt(2.0)); }
static double npdf(double z) { return exp(-0.5 * z * z) / sqrt(2.0 * PI); }

/* G_bottom(v) = int_0^v v' phi(v') dv' with phi = N(u, sig^2) (App. B) */
static double g_bottom(double v, double u, double sg)
{
    double z = (v - u) / sg, z0 = -u / sg;
    return u * (ncdf(z) - ncdf(z0)) + sg * (npdf(z0) - npdf(z));
}

/* G_top(v) = -int_v^0 v' phi(v') dv' for v < 0 (App. B) */
static double g_top(double v, double u, double sg)
{
    double z = (v - u) / sg, z0 = -u / sg;
    return -u * (ncdf(z0) - ncdf(z)) + sg * (npdf(z0) - npdf(z));
}

/* inverse of the flux-weighted CDF by 64 bisection steps on a finite range */
static double sample_vz_bottom(double U, double u, double sg)
{
    double hi = (u > 0 ? u : 0) + 12.0 * sg, lo = 0.0;
    double target = U * g_bottom(hi, u, sg);
    for (int it = 0; it < 64; ++it) {
        double mid = 0.5 * (lo + hi);
        if (g_bottom(mid, u, sg) < target) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

static double sample_vz_top(double U, double u, double sg)
{
    double lo = (u < 0 ? u : 0) - 12.0 * sg, hi = 0.0;
    double target = U * g_top(lo, u, sg);
    for (int it = 0; it < 64; ++it) {
        double mid = 0.5 * (lo + hi);
        if (g_top(mid, u, sg) > target) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------- App. A math */
static const int PA[15] = {0, 1, 0, 1, 2, 0, 2, 1, 3, 0, 2, 3, 1, 4, 0}; /* power of r^2 */
static const int PB[15] = {0, 0, 1, 1, 0, 2, 1, 2, 0, 3, 2, 1, 3, 0, 4}; /* power of z^2 */

static double ipow(double b, int e)
{
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

/* Gauss-Legendre nodes and weights on [-1, 1] from Newton iteration on P_n */
static void gauss_legendre(int n, double* x, double* w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(PI * (i + 0.75) / (n + 0.5)), pp = 1.0;
        for (int iter = 0; iter < 100; ++iter) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= n; ++j) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            double z1 = z;
            z = z1 - p1 / pp;
            if (fabs(z - z1) < 1e-15) {
                /* one more evaluation of the derivative at the converged node */
                p1 = 1.0;
                p2 = 0.0;
                for (int j = 1; j <= n; ++j) {
                    double p3 = p2;
                    p2 = p1;
                    p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
                }
                pp = n * (z * p1 - p2) / (z * z - 1.0);
                break;
            }
        }
        x[i] = -z;
        w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

/* Integral over the cylinder of exp(-|r-r'|/lam)/|r-r'| d^3r' for the field point
 * (r0, 0, z0) inside or on the cylinder.  Written in spherical coordinates centred
 * on the field point, the radial integral is exact:
 *     int_0^S exp(-s/lam) s ds = lam^2 (1 - (1 + S/lam) exp(-S/lam)),
 * with S(theta, phi) the distance to the boundary along the ray.  The angular
 * integral uses Gauss-Legendre on segments where S is smooth: phi in [0, pi/2] and
 * [pi/2, pi] (times 2 for the mirror half), theta split at the two rims. */
static double cyl_integral(double R, double H, double lam, int nq, double r0, double z0)
{
    double* gx = malloc(sizeof(double) * nq);
    double* gw = malloc(sizeof(double) * nq);
    gauss_legendre(nq, gx, gw);
    double hz = 0.5 * H, total = 0.0;
    for (int ps = 0; ps < 2; ++ps) {
        double pa = ps * 0.5 * PI, pbd = pa + 0.5 * PI;
        for (int ip = 0; ip < nq; ++ip) {
            double phi = 0.5 * (pa + pbd) + 0.5 * (pbd - pa) * gx[ip];
            double wphi = 0.5 * (pbd - pa) * gw[ip];
            double c = cos(phi), sn = sin(phi);
            double disc = R * R - r0 * r0 * sn * sn;
            double sh = -r0 * c + sqrt(disc > 0 ? disc : 0.0);
            if (sh < 0) sh = 0;
            double tht = atan2(sh, hz - z0);
            double thb = PI - atan2(sh, hz + z0);
            double edges[4] = {0.0, tht, thb, PI};
            double inner = 0.0;
            for (int seg = 0; seg < 3; ++seg) {
                double ta = edges[seg], tb = edges[seg + 1];
                if (!(tb > ta)) continue;
                for (int it = 0; it < nq; ++it) {
                    double th = 0.5 * (ta + tb) + 0.5 * (tb - ta) * gx[it];
                    double wth = 0.5 * (tb - ta) * gw[it];
                    double S;
                    if (seg == 0) S = (hz - z0) / cos(th);
                    else if (seg == 1) S = sh / sin(th);
                    else S = (hz + z0) / (-cos(th));
                    double xs = S / lam;
                    /* 1 - (1 + x) e^-x; for small x its series sum_{n>=2} (-1)^n (n-1) x^n / n!
                     * avoids the cancellation of the direct form */
                    double f;
                    if (xs < 1e-3) f = xs * xs * (0.5 + xs * (-1.0 / 3.0 + xs * (1.0 / 8.0 + xs * (-1.0 / 30.0))));
                    else f = -expm1(-xs) - xs * exp(-xs);
                    inner += wth * lam * lam * f * sin(th);
                }
            }
            total += wphi * inner;
        }
    }
    free(gx);
    free(gw);
    return 2.0 * total;
}

static double debye_length(const orc_params* p)
{
    double ne = p->Z * p->n_inf; /* quasi-neutral electron density */
    return sqrt(EPS0 * KB * p->T_e / (ne * QE * QE));
}

double orc_cyl_integral(const orc_params* p, double r0, double z0)
{
    return cyl_integral(p->R, p->H, debye_length(p), p->quad_n > 0 ? p->quad_n : 48, r0, z0);
}

/* least squares by Householder QR: A (m x n, row major, overwritten), b (m) -> x (n) */
static int lsq_householder(int m, int n, double* A, double* b, double* x)
{
    for (int k = 0; k < n; ++k) {
        double nrm = 0.0;
        for (int i = k; i < m; ++i) nrm += A[i * n + k] * A[i * n + k];
        nrm = sqrt(nrm);
        if (nrm == 0.0) return -1;
        double alpha = A[k * n + k] > 0 ? -nrm : nrm;
        /* v = a_k - alpha e_k, stored in place */
        A[k * n + k] -= alpha;
        double vnorm2 = 0.0;
        for (int i = k; i < m; ++i) vnorm2 += A[i * n + k] * A[i * n + k];
        for (int j = k + 1; j < n; ++j) {
            double d = 0.0;
            for (int i = k; i < m; ++i) d += A[i * n + k] * A[i * n + j];
            d = 2.0 * d / vnorm2;
            for (int i = k; i < m; ++i) A[i * n + j] -= d * A[i * n + k];
        }
        double d = 0.0;
        for (int i = k; i < m; ++i) d += A[i * n + k] * b[i];
        d = 2.0 * d / vnorm2;
        for (int i = k; i < m; ++i) b[i] -= d * A[i * n + k];
        /* diagonal of R */
        A[k * n + k] = alpha;
    }
    for (int k = n - 1; k >= 0; --k) {
        double s = b[k];
        for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * x[j];
        x[k] = s / A[k * n + k];
    }
    return 0;
}

/* App. A: Phi_ext on the (r, z) grid, then the 15-term fit of Eq. (Polinomial) */
static int fit_eout(orc_state* s)
{
    const orc_params* p = &s->p;
    int nx = p->grid_nx > 0 ? p->grid_nx : 40, nz = p->grid_nz > 0 ? p->grid_nz : 40;
    int nq = p->quad_n > 0 ? p->quad_n : 48;
    int m = (nx + 1) * (nz + 1);
    double* A = malloc(sizeof(double) * m * 15);
    double* b = malloc(sizeof(double) * m);
    double hz = 0.5 * p->H;
    /* potential of the uniform ion fill: charge density Z e n_inf, Yukawa kernel */
    double pref = p->Z * QE * p->n_inf / (4.0 * PI * EPS0);
    int row = 0;
    for (int k = 0; k <= nx; ++k) {
        for (int q = 0; q <= nz; ++q) {
            double r = (double)k / nx * p->R, z = (double)q / nz * hz;
            /* Phi_ext = Phi_0 - Phi_cyl with Phi_0 = 0 (a constant does not change E) */
            b[row] = -pref * cyl_integral(p->R, p->H, s->lam, nq, r, z);
            double rho2 = (r / p->R) * (r / p->R), zeta2 = (z / hz) * (z / hz);
            for (int t = 0; t < 15; ++t) A[row * 15 + t] = ipow(rho2, PA[t]) * ipow(zeta2, PB[t]);
            ++row;
        }
    }
    double beta[15];
    int rc = lsq_householder(m, 15, A, b, beta);
    for (int t = 0; t < 15; ++t) s->alpha[t] = beta[t] / (ipow(p->R * p->R, PA[t]) * ipow(hz * hz, PB[t]));
    free(A);
    free(b);
    return rc;
}

/* E = -grad P (App. A, Eq. extField): E_x = -x (dP/dr)/r, E_z = -z (dP/dz)/z */
static void eout_field(const double* al, double x, double y, double z, double* E)
{
    double r2 = x * x + y * y, z2 = z * z;
    double G = 0.0, K = 0.0;
    for (int t = 0; t < 15; ++t) {
        if (PA[t] >= 1) G += 2.0 * PA[t] * al[t] * ipow(r2, PA[t] - 1) * ipow(z2, PB[t]);
        if (PB[t] >= 1) K += 2.0 * PB[t] * al[t] * ipow(r2, PA[t]) * ipow(z2, PB[t] - 1);
    }
    E[0] = -x * G;
    E[1] = -y * G;
    E[2] = -z * K;
}

void orc_eout(const orc_state* s, double x, double y, double z, double* E) { eout_field(s->alpha, x, y, z, E); }
void orc_alpha(const orc_state* s, double* alpha) { memcpy(alpha, s->alpha, sizeof(double) * 15); }

/* ------------------------------------------------------------------ forces */
/* Accelerations of target ions [i0, i1) and, if f_orbit != NULL, the force of all
 * ions plus E_out on every grain (Eq. 1).  Dust charges are the current Q. */
void orc_forces(const orc_state* s, int64_t i0, int64_t i1, double* acc, double* f_orbit)
{
    const orc_params* p = &s->p;
    const int64_t N = s->N;
    const double lam = s->lam;
    const double k_ii = s->q * s->q / (4.0 * PI * EPS0 * s->m); /* q^2 / (4 pi eps0 m) */
    const double qm = p->Z * QE / p->m_i;                        /* q / m */
    const int ionion = !(p->flags & ORC_F_NO_IONION);
    const int eout = !(p->flags & ORC_F_NO_EOUT);
    const int cut = p->r_cut > 0.0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t i = i0; i < i1; ++i) {
        double ax = 0.0, ay = 0.0, az = 0.0;
        const double xi = s->x[3 * i], yi = s->x[3 * i + 1], zi = s->x[3 * i + 2];
        if (ionion) {
            /* Yukawa pair force with the electron Debye length (Sec. 2) */
            for (int64_t j = 0; j < N; ++j) {
                if (j == i) continue;
                double dx = xi - s->x[3 * j], dy = yi - s->x[3 * j + 1], dz = zi - s->x[3 * j + 2];
                double r = sqrt(dx * dx + dy * dy + dz * dz);
                if (cut && r >= p->r_cut) continue;
                double f = (1.0 + r / lam) * exp(-r / lam) / (r * r * r);
                if (cut && r > p->r_switch) {
                    /* switched energy U S: force -(U' S + U S') r_hat, with U = exp(-r/lam)/r */
                    const double w = p->r_cut - p->r_switch, x = (r - p->r_switch) / w;
                    const double S = 1.0 - x * x * x * (10.0 - 15.0 * x + 6.0 * x * x);
                    const double dS = -30.0 * x * x * (1.0 - x) * (1.0 - x) / w;
                    const double U = exp(-r / lam) / r;
                    f = f * S - U * dS / r;
                }
                ax += f * dx;
                ay += f * dy;
                az += f * dz;
            }
            ax *= k_ii;
            ay *= k_ii;
            az *= k_ii;
        }
        /* bare Coulomb force of each grain on the ion (asymmetric model, Sec. 2) */
        for (int k = 0; k < p->n_dust; ++k) {
            double dx = xi - p->dust[k].x, dy = yi - p->dust[k].y, dz = zi - p->dust[k].z;
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            double c = qm * s->Q[k] / (4.0 * PI * EPS0 * r * r * r);
            ax += c * dx;
            ay += c * dy;
            az += c * dz;
        }
        if (eout) {
            double E[3];
            eout_field(s->alpha, xi, yi, zi, E);
            ax += qm * E[0];
            ay += qm * E[1];
            az += qm * E[2];
        }
        az += qm * s->E; /* driving field along z (Eq. 4's E_ext acting on ions) */
        acc[3 * (i - i0)] = ax;
        acc[3 * (i - i0) + 1] = ay;
        acc[3 * (i - i0) + 2] = az;
    }
    if (f_orbit) {
        for (int k = 0; k < p->n_dust; ++k) {
            /* Eq. 1: q Q_d / (4 pi eps0) sum_i (1 + rho/lam) exp(-rho/lam) (r_d - r_i) / rho^3 + E_out Q_d */
            double sx = 0.0, sy = 0.0, sz = 0.0;
            for (int64_t i = 0; i < N; ++i) {
                double dx = p->dust[k].x - s->x[3 * i], dy = p->dust[k].y - s->x[3 * i + 1],
                       dz = p->dust[k].z - s->x[3 * i + 2];
                double rho = sqrt(dx * dx + dy * dy + dz * dz);
                double f = (1.0 + rho / lam) * exp(-rho / lam) / (rho * rho * rho);
                sx += f * dx;
                sy += f * dy;
                sz += f * dz;
            }
            double c = s->q * s->Q[k] / (4.0 * PI * EPS0);
            double E[3] = {0.0, 0.0, 0.0};
            if (eout) eout_field(s->alpha, p->dust[k].x, p->dust[k].y, p->dust[k].z, E);
            f_orbit[3 * k] = c * sx + E[0] * s->Q[k];
            f_orbit[3 * k + 1] = c * sy + E[1] * s->Q[k];
            f_orbit[3 * k + 2] = c * sz + E[2] * s->Q[k];
        }
    }
}

/* --------------------------------------------------------------- injection */
/* App. B: face by flux probability, position uniform on the face, velocity from the
 * flux-weighted distributions.  Face codes: 0 bottom, 1 top, 2 side. */
void orc_inject_sample(const orc_state* s, uint64_t id, uint32_t step, double* pos, double* vel, int* face)
{
    const orc_params* p = &s->p;
    uint32_t A[4], B[4];
    draw(s, id, step, ST_INJ_A, A);
    draw(s, id, step, ST_INJ_B, B);
    double n0, n1;
    box_muller(B[0], B[1], &n0, &n1);
    if ((uint64_t)A[0] < s->Tbt) {
        int f = (uint64_t)A[0] < s->Tb ? 0 : 1;
        double rho = p->R * sqrt(unif(A[1])), ph = 2.0 * PI * unif(A[2]);
        pos[0] = rho * cos(ph);
        pos[1] = rho * sin(ph);
        pos[2] = f == 0 ? -0.5 * p->H : 0.5 * p->H;
        vel[0] = s->sig * n0;
        vel[1] = s->sig * n1;
        vel[2] = f == 0 ? sample_vz_bottom(unif(A[3]), s->u, s->sig) : sample_vz_top(unif(A[3]), s->u, s->sig);
        *face = f;
    } else {
        double ph = 2.0 * PI * unif(A[1]);
        double c = cos(ph), sn = sin(ph);
        pos[0] = p->R * c;
        pos[1] = p->R * sn;
        pos[2] = p->H * (unif(A[2]) - 0.5);
        /* radial speed from G_side: v_r phi_M(v_r) on v_r > 0, i.e. Rayleigh(sig) */
        double vr = s->sig * sqrt(-2.0 * log(unif(A[3])));
        double vt = (p->flags & ORC_F_PAPER_SIDE) ? 0.0 : s->sig * n0;
        vel[0] = -vr * c - vt * sn;
        vel[1] = -vr * sn + vt * c;
        vel[2] = s->u + s->sig * n1;
        *face = 2;
    }
}

/* ---------------------------------------------------------------- creation */
static int inside_dust(const orc_params* p, double x, double y, double z)
{
    for (int k = 0; k < p->n_dust; ++k) {
        double dx = x - p->dust[k].x, dy = y - p->dust[k].y, dz = z - p->dust[k].z;
        if (dx * dx + dy * dy + dz * dz <= p->dust[k].a * p->dust[k].a) return 1;
    }
    return 0;
}

static void set_err(char* err, int errlen, const char* msg)
{
    if (err && errlen > 0) {
        strncpy(err, msg, errlen - 1);
        err[errlen - 1] = 0;
    }
}

static uint64_t threshold(double prob)
{
    double t = floor(prob * TWO32);
    if (t < 0) t = 0;
    if (t > TWO32) t = TWO32;
    return (uint64_t)t;
}

orc_state* orc_create(const orc_params* pin, char* err, int errlen)
{
    const orc_params* p = pin;
    if (!(p->R > 0 && p->H > 0 && p->dt > 0 && p->m_i > 0 && p->T_e > 0 && p->T_i > 0 && p->n_inf > 0 &&
          p->Z > 0 && p->weight > 0)) {
        set_err(err, errlen, "non-positive physical parameter");
        return NULL;
    }
    if (p->n_dust < 0 || p->n_dust > ORC_MAX_DUST) {
        set_err(err, errlen, "n_dust out of range");
        return NULL;
    }
    if (p->r_cut > 0 && !(p->r_switch >= 0 && p->r_switch < p->r_cut)) {
        set_err(err, errlen, "cutoff: need 0 <= r_switch < r_cut");
        return NULL;
    }
    if (p->mach < 0 || p->E_ext < 0 || p->nu < 0 || (p->mach > 0 && p->E_ext > 0) || (p->E_ext > 0 && p->nu <= 0)) {
        set_err(err, errlen, "flow: give mach or (E_ext with nu > 0)");
        return NULL;
    }
    for (int k = 0; k < p->n_dust; ++k) {
        const orc_dust* d = &p->dust[k];
        if (!(d->a > 0) || sqrt(d->x * d->x + d->y * d->y) + d->a >= p->R || fabs(d->z) + d->a >= 0.5 * p->H) {
            set_err(err, errlen, "dust grain outside the domain");
            return NULL;
        }
    }
    orc_state* s = calloc(1, sizeof(orc_state));
    s->p = *p;
    if (s->p.T_n <= 0) s->p.T_n = s->p.T_i;
    p = &s->p;
    s->lam = debye_length(p);
    s->cs = sqrt(p->Z * KB * p->T_e / p->m_i);
    s->sig = sqrt(KB * p->T_i / p->m_i);
    s->sig_n = sqrt(KB * p->T_n / p->m_i);
    s->q = p->weight * p->Z * QE;
    s->m = p->weight * p->m_i;
    if (p->mach > 0) {
        s->u = p->mach * s->cs;
        /* field-driven collisional flow: drift u = Z e E / (m_i nu) (Table 3 reading) */
        s->E = p->nu > 0 ? p->m_i * p->nu * s->u / (p->Z * QE) : 0.0;
    } else if (p->E_ext > 0) {
        s->E = p->E_ext;
        s->u = p->Z * QE * p->E_ext / (p->m_i * p->nu);
    }
    /* App. B fluxes for phi(v_z) = N(u, sig^2), phi_M = N(0, sig^2) */
    double zu = s->u / s->sig;
    double Jb = PI * p->R * p->R * (s->u * ncdf(zu) + s->sig * npdf(zu));
    double Jt = PI * p->R * p->R * (-s->u * ncdf(-zu) + s->sig * npdf(zu));
    double Js = 2.0 * PI * p->R * p->H * s->sig / sqrt(2.0 * PI);
    double J = Jb + Jt + Js;
    s->inj_rate = p->n_inf / p->weight * J;
    s->pb = Jb / J;
    s->pt = Jt / J;
    s->ps = Js / J;
    s->Tb = threshold(s->pb);
    s->Tbt = threshold(s->pb + s->pt);
    s->pcoll = -expm1(-p->nu * p->dt);
    s->Tcoll = threshold(s->pcoll);
    /* OML electron flux at zero potential: n_e sqrt(8 k T_e / (pi m_e)) / 4 per unit area */
    s->Ie0 = p->Z * p->n_inf * sqrt(8.0 * KB * p->T_e / (PI * ME)) / 4.0;
    if (p->has_alpha) memcpy(s->alpha, p->alpha, sizeof(double) * 15);
    else if (!(p->flags & ORC_F_NO_EOUT)) {
        if (fit_eout(s)) {
            set_err(err, errlen, "E_out fit failed");
            free(s);
            return NULL;
        }
    }
    int64_t N = p->n_ions > 0 ? p->n_ions : (int64_t)llround(p->n_inf * PI * p->R * p->R * p->H / p->weight);
    s->N = N;
    s->x = malloc(sizeof(double) * 3 * (N > 0 ? N : 1));
    s->v = malloc(sizeof(double) * 3 * (N > 0 ? N : 1));
    s->a = malloc(sizeof(double) * 3 * (N > 0 ? N : 1));
    s->id = malloc(sizeof(uint64_t) * (N > 0 ? N : 1));
    for (int k = 0; k < p->n_dust; ++k) s->Q[k] = p->dust[k].q0;
    /* initial fill: uniform in the cylinder outside the grains, shifted Maxwellian */
    for (int64_t i = 0; i < N; ++i) {
        uint32_t w[4];
        int ok = 0;
        for (uint32_t att = 0; att < 4096 && !ok; ++att) {
            draw(s, (uint64_t)i, att, ST_INIT_POS, w);
            double rho = p->R * sqrt(unif(w[0])), ph = 2.0 * PI * unif(w[1]);
            double x = rho * cos(ph), y = rho * sin(ph), z = p->H * (unif(w[2]) - 0.5);
            if (!inside_dust(p, x, y, z)) {
                s->x[3 * i] = x;
                s->x[3 * i + 1] = y;
                s->x[3 * i + 2] = z;
                ok = 1;
            }
        }
        if (!ok) {
            set_err(err, errlen, "initial placement failed");
            orc_destroy(s);
            return NULL;
        }
        draw(s, (uint64_t)i, 0, ST_INIT_VEL, w);
        double n0, n1, n2, n3;
        box_muller(w[0], w[1], &n0, &n1);
        box_muller(w[2], w[3], &n2, &n3);
        s->v[3 * i] = s->sig * n0;
        s->v[3 * i + 1] = s->sig * n1;
        s->v[3 * i + 2] = s->u + s->sig * n2;
        s->id[i] = (uint64_t)i;
    }
    s->next_id = N;
    s->step = 0;
    orc_forces(s, 0, N, s->a, NULL);
    return s;
}

void orc_destroy(orc_state* s)
{
    if (!s) return;
    free(s->x);
    free(s->v);
    free(s->a);
    free(s->id);
    free(s->rec);
    free(s->ev);
    free(s);
}

int64_t orc_num_ions(const orc_state* s) { return s->N; }
int64_t orc_step_index(const orc_state* s) { return s->step; }

void orc_get_ions(const orc_state* s, double* x, double* v, double* a, uint64_t* id)
{
    if (x) memcpy(x, s->x, sizeof(double) * 3 * s->N);
    if (v) memcpy(v, s->v, sizeof(double) * 3 * s->N);
    if (a) memcpy(a, s->a, sizeof(double) * 3 * s->N);
    if (id) memcpy(id, s->id, sizeof(uint64_t) * s->N);
}

int orc_set_ions(orc_state* s, int64_t n, const double* x, const double* v, const uint64_t* id, int64_t next_id)
{
    if (n < 0) return -1;
    size_t cnt = n > 0 ? (size_t)n : 1;
    s->x = realloc(s->x, sizeof(double) * 3 * cnt);
    s->v = realloc(s->v, sizeof(double) * 3 * cnt);
    s->a = realloc(s->a, sizeof(double) * 3 * cnt);
    s->id = realloc(s->id, sizeof(uint64_t) * cnt);
    s->N = n;
    memcpy(s->x, x, sizeof(double) * 3 * n);
    memcpy(s->v, v, sizeof(double) * 3 * n);
    memcpy(s->id, id, sizeof(uint64_t) * n);
    s->next_id = next_id;
    orc_forces(s, 0, n, s->a, NULL);
    return 0;
}

/* replace the ion state without evaluating forces (accelerations set to zero): for
 * sampled force checks at sizes where the full O(N^2) pass is too slow */
int orc_load_ions(orc_state* s, int64_t n, const double* x, const double* v, const uint64_t* id, int64_t next_id)
{
    if (n < 0) return -1;
    size_t cnt = n > 0 ? (size_t)n : 1;
    s->x = realloc(s->x, sizeof(double) * 3 * cnt);
    s->v = realloc(s->v, sizeof(double) * 3 * cnt);
    s->a = realloc(s->a, sizeof(double) * 3 * cnt);
    s->id = realloc(s->id, sizeof(uint64_t) * cnt);
    s->N = n;
    memcpy(s->x, x, sizeof(double) * 3 * n);
    memcpy(s->v, v, sizeof(double) * 3 * n);
    memcpy(s->id, id, sizeof(uint64_t) * n);
    memset(s->a, 0, sizeof(double) * 3 * n);
    s->next_id = next_id;
    return 0;
}

void orc_derived(const orc_state* s, double* o)
{
    o[0] = s->lam;
    o[1] = s->cs;
    o[2] = s->sig;
    o[3] = s->sig_n;
    o[4] = s->u;
    o[5] = s->E;
    o[6] = s->q;
    o[7] = s->m;
    o[8] = s->pb;
    o[9] = s->pt;
    o[10] = s->ps;
    o[11] = (double)s->Tb;
    o[12] = (double)s->Tbt;
    o[13] = (double)s->Tcoll;
    o[14] = (double)s->N;
    o[15] = s->Ie0;
    o[16] = s->pcoll;
    o[17] = (double)s->next_id;
    for (int i = 18; i < 24; ++i) o[i] = 0.0;
}

/* electron flux onto grain k (OML, Sec. 2 "consistent" model), electrons per second */
static double electron_flux(const orc_state* s, int k, double Q)
{
    double a = s->p.dust[k].a;
    double phi = Q / (4.0 * PI * EPS0 * a); /* isolated-sphere capacitance */
    double x = QE * phi / (KB * s->p.T_e);
    double fac = x <= 0 ? exp(x) : 1.0 + x;
    return 4.0 * PI * a * a * s->Ie0 * fac;
}

static void grow_records(orc_state* s, int64_t need)
{
    if (need <= s->cap) return;
    int64_t nc = s->cap ? s->cap : 256;
    while (nc < need) nc *= 2;
    s->rec = realloc(s->rec, sizeof(double) * ORC_MAX_DUST * ORC_REC * nc);
    s->ev = realloc(s->ev, sizeof(int32_t) * ORC_EV * nc);
    memset(s->rec + ORC_MAX_DUST * ORC_REC * s->cap, 0, sizeof(double) * ORC_MAX_DUST * ORC_REC * (nc - s->cap));
    memset(s->ev + ORC_EV * s->cap, 0, sizeof(int32_t) * ORC_EV * (nc - s->cap));
    s->cap = nc;
}

/* one time step s -> s+1 in the canonical order */
/* Number of superions injected in a step when the count follows the fluxes: Poisson
 * with mean lam = inj_rate dt.  lam is split into chunks of at most 64; each chunk is
 * drawn by inversion, summing e^-l l^x / x! in increasing x until the sum reaches one
 * uniform U = (w + 1/2) 2^-32.  Uniform j of step s is word j mod 4 of the Philox block
 * with counter (j / 4, 0, s, stream 6). */
static int64_t poisson_injections(const orc_state* s, uint32_t sn)
{
    double rem = s->inj_rate * s->p.dt;
    int64_t k = 0;
    for (int j = 0; rem > 0.0; ++j) {
        const double l = rem > 64.0 ? 64.0 : rem;
        rem -= l;
        uint32_t w[4];
        draw(s, (uint64_t)(j >> 2), sn, ST_INJ_N, w);
        const double U = unif(w[j & 3]);
        double pr = exp(-l), F = pr;
        int64_t x = 0;
        while (U > F && x < 100000) {
            ++x;
            pr = pr * (l / (double)x);
            F += pr;
        }
        k += x;
    }
    return k;
}

int64_t orc_injections(const orc_state* s, uint32_t step) { return poisson_injections(s, step); }

static void step_once(orc_state* s)
{
    const orc_params* p = &s->p;
    const int64_t N = s->N;
    const double dt = p->dt;
    const uint32_t sn = (uint32_t)(s->step + 1);
    const int D = p->n_dust;
    grow_records(s, s->step + 1);
    double* rec = s->rec + (size_t)s->step * ORC_MAX_DUST * ORC_REC;
    int32_t* ev = s->ev + (size_t)s->step * ORC_EV;

    /* 1. first half kick and drift (velocity Verlet) */
    for (int64_t i = 0; i < 3 * N; ++i) {
        s->v[i] += 0.5 * dt * s->a[i];
        s->x[i] += dt * s->v[i];
    }
    /* 2. absorption (lowest grain index wins) then outflow, in ion order */
    int* cls = malloc(sizeof(int) * (N > 0 ? N : 1));
    int64_t nabs[ORC_MAX_DUST] = {0};
    double P[ORC_MAX_DUST][3] = {{0}};
    int64_t nout = 0;
    for (int64_t i = 0; i < N; ++i) {
        double x = s->x[3 * i], y = s->x[3 * i + 1], z = s->x[3 * i + 2];
        cls[i] = -2;
        if (!(p->flags & ORC_F_NO_ABSORB)) {
            for (int k = 0; k < D; ++k) {
                double dx = x - p->dust[k].x, dy = y - p->dust[k].y, dz = z - p->dust[k].z;
                if (dx * dx + dy * dy + dz * dz <= p->dust[k].a * p->dust[k].a) {
                    cls[i] = k;
                    break;
                }
            }
        }
        if (cls[i] == -2 && !(p->flags & ORC_F_NO_BOUNDARY)) {
            if (x * x + y * y > p->R * p->R || fabs(z) > 0.5 * p->H) cls[i] = -1;
        }
        if (cls[i] >= 0) {
            int k = cls[i];
            nabs[k] += 1;
            /* Eq. 3 with the superion mass and the half-step velocity that carried it in */
            P[k][0] += s->m * s->v[3 * i];
            P[k][1] += s->m * s->v[3 * i + 1];
            P[k][2] += s->m * s->v[3 * i + 2];
        } else if (cls[i] == -1) {
            nout += 1;
        }
    }
    /* 3. stable compaction of survivors, then 1:1 re-injection at the end (App. B) */
    int64_t w = 0;
    for (int64_t i = 0; i < N; ++i) {
        if (cls[i] != -2) continue;
        if (w != i) {
            for (int c = 0; c < 3; ++c) {
                s->x[3 * w + c] = s->x[3 * i + c];
                s->v[3 * w + c] = s->v[3 * i + c];
            }
            s->id[w] = s->id[i];
        }
        ++w;
    }
    int64_t removed = N - w;
    /* 1:1 replacement keeps N; with the flux rule a Poisson count enters instead */
    const int64_t nin = (p->flags & ORC_F_FLUX_INJECT) ? poisson_injections(s, sn) : removed;
    if (w + nin > N) {
        const int64_t cnt = w + nin;
        s->x = realloc(s->x, sizeof(double) * 3 * cnt);
        s->v = realloc(s->v, sizeof(double) * 3 * cnt);
        s->a = realloc(s->a, sizeof(double) * 3 * cnt);
        s->id = realloc(s->id, sizeof(uint64_t) * cnt);
    }
    int64_t inj[3] = {0, 0, 0};
    for (int64_t r = 0; r < nin; ++r) {
        uint64_t nid = (uint64_t)(s->next_id + r);
        int face;
        orc_inject_sample(s, nid, sn, &s->x[3 * (w + r)], &s->v[3 * (w + r)], &face);
        s->id[w + r] = nid;
        inj[face] += 1;
    }
    s->next_id += nin;
    s->N = w + nin;
    free(cls);

    /* 4. forces at the new positions, with the charges of the previous step */
    double fo[ORC_MAX_DUST * 3];
    orc_forces(s, 0, s->N, s->a, fo);

    /* 5. second half kick; 6. Andersen collisions with neutrals (Sec. 2) */
    int64_t ncoll = 0;
    for (int64_t i = 0; i < s->N; ++i) {
        for (int c = 0; c < 3; ++c) s->v[3 * i + c] += 0.5 * dt * s->a[3 * i + c];
        uint32_t wd[4];
        draw(s, s->id[i], sn, ST_COLL, wd);
        if ((uint64_t)wd[0] < s->Tcoll) {
            uint32_t wv[4];
            double n0, n1, n2, n3;
            draw(s, s->id[i], sn, ST_COLL_VEL, wv);
            box_muller(wv[0], wv[1], &n0, &n1);
            box_muller(wv[2], wv[3], &n2, &n3);
            s->v[3 * i] = s->sig_n * n0;
            s->v[3 * i + 1] = s->sig_n * n1;
            s->v[3 * i + 2] = s->sig_n * n2;
            ++ncoll;
        }
    }

    /* 7. dust: force terms with Q^s (Eqs. 1-4), then the charge update */
    for (int k = 0; k < D; ++k) {
        double* r = rec + k * ORC_REC;
        double fdd[3] = {0.0, 0.0, 0.0};
        for (int q = 0; q < D; ++q) {
            if (q == k) continue;
            double dx = p->dust[k].x - p->dust[q].x, dy = p->dust[k].y - p->dust[q].y, dz = p->dust[k].z - p->dust[q].z;
            double d = sqrt(dx * dx + dy * dy + dz * dz);
            double c = s->Q[k] * s->Q[q] / (4.0 * PI * EPS0 * d * d * d);
            fdd[0] += c * dx;
            fdd[1] += c * dy;
            fdd[2] += c * dz;
        }
        for (int c = 0; c < 3; ++c) {
            r[1 + c] = fo[3 * k + c];
            r[4 + c] = fdd[c];
            r[7 + c] = P[k][c] / dt;
        }
        r[10] = 0.0;
        r[11] = 0.0;
        r[12] = s->Q[k] * s->E;
    }
    for (int k = 0; k < D; ++k) {
        if (p->charge_model == ORC_Q_CONSISTENT) {
            double Qn = s->Q[k] + s->q * (double)nabs[k] - QE * electron_flux(s, k, s->Q[k]) * dt;
            s->Q[k] = Qn;
        }
        rec[k * ORC_REC] = s->Q[k];
    }
    for (int k = 0; k < ORC_MAX_DUST; ++k) ev[k] = k < D ? (int32_t)nabs[k] : 0;
    ev[8] = (int32_t)nout;
    ev[9] = (int32_t)inj[0];
    ev[10] = (int32_t)inj[1];
    ev[11] = (int32_t)inj[2];
    ev[12] = (int32_t)ncoll;
    s->step += 1;
}

int orc_step(orc_state* s, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) step_once(s);
    return 0;
}

void orc_records(const orc_state* s, int64_t first, int64_t count, double* rec, int32_t* ev)
{
    /* first is the 1-based step index of the first record */
    for (int64_t t = 0; t < count; ++t) {
        int64_t idx = first - 1 + t;
        if (rec) memcpy(rec + t * ORC_MAX_DUST * ORC_REC, s->rec + idx * ORC_MAX_DUST * ORC_REC,
                        sizeof(double) * ORC_MAX_DUST * ORC_REC);
        if (ev) memcpy(ev + t * ORC_EV, s->ev + idx * ORC_EV, sizeof(int32_t) * ORC_EV);
    }
}

void orc_dust_q(const orc_state* s, double* q)
{
    for (int k = 0; k < s->p.n_dust; ++k) q[k] = s->Q[k];
}

/* window means over records avg_start..step and batch-means standard errors
 * (20 equal batches of the window) for every record entry */
int orc_dust_terms(const orc_state* s, double* mean, double* se)
{
    int64_t first = s->p.avg_start > 0 ? s->p.avg_start : 1;
    int64_t cnt = s->step - first + 1;
    int D = s->p.n_dust;
    for (int k = 0; k < D; ++k)
        for (int c = 0; c < ORC_REC; ++c) {
            double sum = 0.0;
            for (int64_t t = 0; t < cnt; ++t) sum += s->rec[(first - 1 + t) * ORC_MAX_DUST * ORC_REC + k * ORC_REC + c];
            mean[k * ORC_REC + c] = cnt > 0 ? sum / cnt : NAN;
            double sev = NAN;
            int64_t bl = cnt / 20;
            if (bl >= 1) {
                double bm[20], mu = 0.0;
                for (int b = 0; b < 20; ++b) {
                    double bs = 0.0;
                    for (int64_t t = 0; t < bl; ++t)
                        bs += s->rec[(first - 1 + b * bl + t) * ORC_MAX_DUST * ORC_REC + k * ORC_REC + c];
                    bm[b] = bs / bl;
                    mu += bm[b] / 20.0;
                }
                double var = 0.0;
                for (int b = 0; b < 20; ++b) var += (bm[b] - mu) * (bm[b] - mu);
                sev = sqrt(var / 19.0 / 20.0);
            }
            se[k * ORC_REC + c] = sev;
        }
    return cnt > 0 ? 0 : -1;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
