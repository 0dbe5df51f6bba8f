// Host side of the GB300 ion-flow-around-dust library: the C ABI of opendust.h.
//
// od_create validates the parameters (before any device work), derives the plasma
// constants, builds the App. A cavity field (device quadrature + host least squares),
// plans the pair-kernel partition, allocates device memory and places the initial
// ions; od_step replays a captured graph of one step (or launches its kernels
// directly in profiling mode).
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "od_host.h"

using namespace od;
using namespace od::host;

namespace od {
namespace host {

thread_local std::string g_create_error;


double norm_cdf(double z) { return 0.5 * std::erfc(-z / std::sqrt(2.0)); }
double norm_pdf(double z) { return std::exp(-0.5 * z * z) / std::sqrt(2.0 * kPI); }

unsigned long long prob_threshold(double p)
{
    double t = std::floor(p * kTWO32);
    t = std::min(std::max(t, 0.0), kTWO32);
    return (unsigned long long)t;
}

// App. B flux integrals of the axial distribution N(u, s^2) through the bottom face up
// to speed v >= 0, and through the top face from speed v <= 0 up to 0
double flux_bottom_h(double v, double u, double s)
{
    const double z = (v - u) / s, z0 = -u / s;
    return u * (norm_cdf(z) - norm_cdf(z0)) + s * (norm_pdf(z0) - norm_pdf(z));
}

double flux_top_h(double v, double u, double s)
{
    const double z = (v - u) / s, z0 = -u / s;
    return -u * (norm_cdf(z0) - norm_cdf(z)) + s * (norm_pdf(z0) - norm_pdf(z));
}

// inverse flux CDFs at U = k / VTAB_K for both faces (bisection to FP64 resolution);
// layout: bottom [0..K], top [K+1..2K+1]
void build_vtab(double u, double s, std::vector<double>& tab, double& gmax_b, double& gmax_t)
{
    const int K = VTAB_K;
    tab.assign(2 * (K + 1), 0.0);
    const double vb = std::max(u, 0.0) + 12.0 * s;
    gmax_b = flux_bottom_h(vb, u, s);
    for (int k = 0; k <= K; ++k) {
        const double target = (double)k / K * gmax_b;
        double lo = k > 0 ? tab[k - 1] : 0.0, hi = vb;
        for (int it = 0; it < 200 && hi - lo > 1e-15 * vb; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (flux_bottom_h(mid, u, s) < target) lo = mid;
            else hi = mid;
        }
        tab[k] = k == K ? vb : 0.5 * (lo + hi);
    }
    const double vt = std::min(u, 0.0) - 12.0 * s;
    gmax_t = flux_top_h(vt, u, s);
    double* tt = tab.data() + K + 1;
    for (int k = 0; k <= K; ++k) {
        const double target = (double)k / K * gmax_t;
        double lo = vt, hi = k > 0 ? tt[k - 1] : 0.0;
        for (int it = 0; it < 200 && hi - lo > 1e-15 * (-vt); ++it) {
            const double mid = 0.5 * (lo + hi);
            if (flux_top_h(mid, u, s) > target) lo = mid;
            else hi = mid;
        }
        tt[k] = k == K ? vt : 0.5 * (lo + hi);
    }
}

void gl_nodes(int n, std::vector<double>& x, std::vector<double>& w);

// OML currents onto an isolated sphere of radius a at potential phi <= 0 (Sec. 2 "oml"
// charging): electrons repelled (Boltzmann factor), ions attracted with the orbital
// cross-section pi a^2 (1 - 2 Z e phi / (m v^2)) from a Maxwellian of thermal speed sig
// drifting at u.  The ion current is one speed integral of v^3 sigma(v) times the angular
// average of the shifted Maxwellian, done by Gauss-Legendre on [0, u] and [u, u + 14 sig].
double oml_ion_current(double a, double phi, double n, double m, double sig, double u, double Z)
{
    static std::vector<double> gx, gw;
    if (gx.empty()) gl_nodes(96, gx, gw);
    auto integrand = [&](double v) {
        if (v <= 0.0) return 0.0;
        const double cross = kPI * a * a * (1.0 - 2.0 * Z * kQE * phi / (m * v * v));
        double ang;
        if (u <= 0.0) {
            ang = 4.0 * kPI * std::exp(-v * v / (2.0 * sig * sig));
        } else {
            const double x = v * u / (sig * sig);
            ang = 2.0 * kPI * (std::exp(-(v - u) * (v - u) / (2 * sig * sig)) - std::exp(-(v + u) * (v + u) / (2 * sig * sig))) / x;
        }
        return v * v * v * cross * ang;
    };
    const double edges[3] = {0.0, u > 0.0 ? u : 0.0, (u > 0.0 ? u : 0.0) + 14.0 * sig};
    double total = 0.0;
    for (int s = 0; s < 2; ++s) {
        const double lo = edges[s], hi = edges[s + 1];
        if (!(hi > lo)) continue;
        for (size_t i = 0; i < gx.size(); ++i) total += 0.5 * (hi - lo) * gw[i] * integrand(0.5 * (lo + hi) + 0.5 * (hi - lo) * gx[i]);
    }
    return Z * kQE * n * total * std::pow(2.0 * kPI * sig * sig, -1.5);
}

// OML floating charge (C): I_ion(phi) = I_electron(phi) by bisection on phi in
// [-200 k T_e / e, 0], Q = 4 pi eps0 a phi
double oml_charge(const od_params* p, double a)
{
    const double Z = p->ion_charge_number;
    const double sig = std::sqrt(kKB * p->T_i / p->ion_mass);
    double u = 0.0;
    if (p->mach > 0) u = p->mach * std::sqrt(Z * kKB * p->T_e / p->ion_mass);
    else if (p->E_ext > 0 && p->nu_in > 0) u = Z * kQE * p->E_ext / (p->ion_mass * p->nu_in);
    const double ne = Z * p->n_inf;
    auto net = [&](double phi) {
        const double ie = kQE * ne * kPI * a * a * std::sqrt(8.0 * kKB * p->T_e / (kPI * kME)) * std::exp(kQE * phi / (kKB * p->T_e));
        return oml_ion_current(a, phi, p->n_inf, p->ion_mass, sig, u, Z) - ie;
    };
    double lo = -200.0 * kKB * p->T_e / kQE, hi = 0.0;  // net(lo) > 0 > net(hi)
    for (int it = 0; it < 200 && hi - lo > 1e-14 * kKB * p->T_e / kQE; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (net(mid) > 0.0) lo = mid;
        else hi = mid;
    }
    return 4.0 * kPI * kEPS0 * a * 0.5 * (lo + hi);
}

// paper's monomial order of Eq. (Polinomial): alpha_t multiplies r^(2 a_t) z^(2 b_t)
const int kPowR[15] = {0, 1, 0, 1, 2, 0, 2, 1, 3, 0, 2, 3, 1, 4, 0};
const int kPowZ[15] = {0, 0, 1, 1, 0, 2, 1, 2, 0, 3, 2, 1, 3, 0, 4};

// index of r2^p z2^q among the 10 monomials of degree <= 3 used by the device field
int mono_index(int p, int q)
{
    static const int tab[4][4] = {{0, 2, 5, 9}, {1, 4, 8, -1}, {3, 7, -1, -1}, {6, -1, -1, -1}};
    return tab[p][q];
}

// Gauss-Legendre nodes/weights on [-1, 1] (Newton on the three-term recurrence)
void gl_nodes(int n, std::vector<double>& x, std::vector<double>& w)
{
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double t = std::cos(kPI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) {
                p1 = t;
                p0 = 1.0;
            }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
            const double dt = p1 / dp;
            t -= dt;
            if (std::fabs(dt) < 1e-16) break;
        }
        double p0 = 1.0, p1 = t;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (t * p1 - p0) / (t * t - 1.0);
        x[i] = t;
        w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

// least squares min |A c - b| by modified Gram-Schmidt on [A | b] (column-major A: m x n)
bool lsq_mgs(int m, int n, std::vector<double> A, std::vector<double> b, double* c)
{
    std::vector<double> R(n * n, 0.0), z(n, 0.0);
    for (int j = 0; j < n; ++j) {
        double* aj = &A[(size_t)j * m];
        double nr = 0.0;
        for (int i = 0; i < m; ++i) nr += aj[i] * aj[i];
        nr = std::sqrt(nr);
        if (!(nr > 0.0)) return false;
        R[j * n + j] = nr;
        for (int i = 0; i < m; ++i) aj[i] /= nr;
        for (int k = j + 1; k < n; ++k) {
            double* ak = &A[(size_t)k * m];
            double d = 0.0;
            for (int i = 0; i < m; ++i) d += aj[i] * ak[i];
            R[j * n + k] = d;
            for (int i = 0; i < m; ++i) ak[i] -= d * aj[i];
        }
        double d = 0.0;
        for (int i = 0; i < m; ++i) d += aj[i] * b[i];
        z[j] = d;
        for (int i = 0; i < m; ++i) b[i] -= d * aj[i];
    }
    for (int j = n - 1; j >= 0; --j) {
        double s = z[j];
        for (int k = j + 1; k < n; ++k) s -= R[j * n + k] * c[k];
        c[j] = s / R[j * n + j];
    }
    return true;
}

}  // namespace host
}  // namespace od

void od::set_global_error(const std::string& msg) { g_create_error = msg; }

namespace od {
namespace host {

int fail(od_handle* h, int code, const std::string& msg)
{
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

int cuda_fail(od_handle* h, cudaError_t e, const char* where)
{
    return fail(h, e == cudaErrorMemoryAllocation ? OD_ENOMEM : OD_ECUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}


// parameter checks that need no device
int validate(const od_params* p, std::string& msg)
{
    if (!p) {
        msg = "params is NULL";
        return OD_EINVAL;
    }
    auto pos = [](double v) { return std::isfinite(v) && v > 0.0; };
    if (!(pos(p->ion_mass) && pos(p->ion_charge_number) && pos(p->T_i) && pos(p->T_e) && pos(p->n_inf) &&
          pos(p->R) && pos(p->H) && pos(p->dt) && pos(p->weight))) {
        msg = "ion_mass, ion_charge_number, T_i, T_e, n_inf, R, H, dt and weight must be finite and > 0";
        return OD_EINVAL;
    }
    if (!(std::isfinite(p->mach) && std::isfinite(p->E_ext) && std::isfinite(p->nu_in) && p->mach >= 0 &&
          p->E_ext >= 0 && p->nu_in >= 0)) {
        msg = "mach, E_ext and nu_in must be finite and >= 0";
        return OD_EINVAL;
    }
    if (p->mach > 0 && p->E_ext > 0) {
        msg = "give either mach or E_ext, not both";
        return OD_EINVAL;
    }
    if (p->E_ext > 0 && !(p->nu_in > 0)) {
        msg = "a field-driven flow (E_ext > 0) needs nu_in > 0";
        return OD_EINVAL;
    }
    if (p->n_dust < 0 || p->n_dust > OD_MAX_DUST) {
        msg = "n_dust must be in 0..8";
        return OD_EINVAL;
    }
    if (p->n_dust > 0 && !p->dust) {
        msg = "dust is NULL with n_dust > 0";
        return OD_EINVAL;
    }
    for (int k = 0; k < p->n_dust; ++k) {
        const od_dust& d = p->dust[k];
        if (!(pos(d.radius) && std::isfinite(d.x) && std::isfinite(d.y) && std::isfinite(d.z) && std::isfinite(d.q0))) {
            msg = "grain " + std::to_string(k) + ": radius must be > 0 and all values finite";
            return OD_EINVAL;
        }
        if (std::sqrt(d.x * d.x + d.y * d.y) + d.radius >= p->R || std::fabs(d.z) + d.radius >= 0.5 * p->H) {
            msg = "grain " + std::to_string(k) + " does not lie inside the cylinder";
            return OD_EINVAL;
        }
    }
    if (p->charge_model != OD_Q_GIVEN && p->charge_model != OD_Q_CONSISTENT && p->charge_model != OD_Q_OML) {
        msg = "charge_model must be OD_Q_GIVEN, OD_Q_CONSISTENT or OD_Q_OML";
        return OD_EINVAL;
    }
    if (p->n_ions < 0) {
        msg = "n_ions must be >= 0";
        return OD_EINVAL;
    }
    const double nreq = p->n_ions > 0 ? (double)p->n_ions : p->n_inf * kPI * p->R * p->R * p->H / p->weight;
    if (!(nreq < 2.0e8)) {
        msg = "too many ions (limit 2e8 per run)";
        return OD_EINVAL;
    }
    {
        // far-away padding of the pair kernels sits at 3e4 scaled units (r log2(e) / lambda_De)
        const double lam = std::sqrt(kEPS0 * kKB * p->T_e / (p->ion_charge_number * p->n_inf * kQE * kQE));
        if (std::sqrt(p->R * p->R + 0.25 * p->H * p->H) * 1.4426950408889634 / lam > 1e4) {
            msg = "domain larger than 6,900 electron Debye lengths";
            return OD_EINVAL;
        }
    }
    if (p->eout_grid < 0 || p->eout_grid > 400) {
        msg = "eout_grid must be in 0..400";
        return OD_EINVAL;
    }
    return OD_OK;
}

// derived constants of Sec. 2 and App. B; N from the density when n_ions == 0
void derive(const od_params* p, Phys& P, od_handle* h)
{
    const double Z = p->ion_charge_number;
    const double Tn = p->T_n > 0 ? p->T_n : p->T_i;
    const double lam = std::sqrt(kEPS0 * kKB * p->T_e / (Z * p->n_inf * kQE * kQE));
    const double cs = std::sqrt(Z * kKB * p->T_e / p->ion_mass);
    P.sig = std::sqrt(kKB * p->T_i / p->ion_mass);
    P.sig_n = std::sqrt(kKB * Tn / p->ion_mass);
    P.q = p->weight * Z * kQE;
    P.m = p->weight * p->ion_mass;
    P.u = 0.0;
    P.E = 0.0;
    if (p->mach > 0) {
        P.u = p->mach * cs;
        if (p->nu_in > 0) P.E = p->ion_mass * p->nu_in * P.u / (Z * kQE);
    } else if (p->E_ext > 0) {
        P.E = p->E_ext;
        P.u = Z * kQE * p->E_ext / (p->ion_mass * p->nu_in);
    }
    const double zu = P.u / P.sig;
    const double Jb = kPI * p->R * p->R * (P.u * norm_cdf(zu) + P.sig * norm_pdf(zu));
    const double Jt = kPI * p->R * p->R * (-P.u * norm_cdf(-zu) + P.sig * norm_pdf(zu));
    const double Js = 2.0 * kPI * p->R * p->H * P.sig / std::sqrt(2.0 * kPI);
    const double J = Jb + Jt + Js;
    P.inj_lambda = p->n_inf / p->weight * J * p->dt;
    P.inj_ahead_flux = (int)std::min((double)INJ_AHEAD, std::ceil(P.inj_lambda + 6.0 * std::sqrt(P.inj_lambda)) + 32.0);
    P.Tb = prob_threshold(Jb / J);
    P.Tbt = prob_threshold((Jb + Jt) / J);
    const double pc = -std::expm1(-p->nu_in * p->dt);
    P.Tcoll = prob_threshold(pc);
    P.dt = p->dt;
    P.R = p->R;
    P.H = p->H;
    P.hz = 0.5 * p->H;
    P.R2 = p->R * p->R;
    P.qm = Z * kQE / p->ion_mass;
    P.kdi = Z * kQE / (4.0 * kPI * kEPS0 * p->ion_mass);
    P.korb = P.q / (4.0 * kPI * kEPS0);
    P.inv4pieps0 = 1.0 / (4.0 * kPI * kEPS0);
    P.lam_inv = 1.0 / lam;
    const double Ls = lam / 1.4426950408889634;  // lambda / log2(e)
    P.Ls_inv = (float)(1.0 / Ls);
    P.k_ii = (float)(P.q * P.q / (4.0 * kPI * kEPS0 * P.m * Ls * Ls));
    P.key0 = (uint32_t)(p->seed & 0xffffffffull);
    P.key1 = (uint32_t)(p->seed >> 32);
    P.D = p->n_dust;
    for (int k = 0; k < p->n_dust; ++k) {
        P.gx[k] = p->dust[k].x;
        P.gy[k] = p->dust[k].y;
        P.gz[k] = p->dust[k].z;
        P.ga[k] = p->dust[k].radius;
        P.ga2[k] = p->dust[k].radius * p->dust[k].radius;
    }
    P.flags = p->flags;
    P.charge_model = p->charge_model;
    P.avg_start = p->avg_start > 0 ? p->avg_start : 1;
    P.Ie0 = Z * p->n_inf * std::sqrt(8.0 * kKB * p->T_e / (kPI * kME)) / 4.0;
    P.e_over_kTe = kQE / (kKB * p->T_e);
    P.spin_limit = SPIN_LIMIT;
    P.test_hold_tile0 = 0;
    const long long N = p->n_ions > 0 ? p->n_ions : std::llround(p->n_inf * kPI * p->R * p->R * p->H / p->weight);
    P.N = (int)N;
    // Scaled units s = r / Ls.  Term sum of an ion at the centre of a uniform fill (its pair
    // terms summed without signs), over the largest centred sphere of radius L: 4 pi n_s
    // int_0^L (1 + s ln2) 2^-s ds, n_s the ions per unit scaled volume.  The fixed-point
    // grid of the symmetric pair sums is 2^-30 of it (power of two).
    P.ls_inv = 1.0 / Ls;
    const double Rs = p->R / Ls, Hs = 0.5 * p->H / Ls;
    const double n_s = (double)std::max(N, 1ll) / (kPI * p->R * p->R * p->H) * Ls * Ls * Ls;
    const double L = std::min(Rs, Hs), ln2 = 0.69314718055994531;
    const double ts = 4.0 * kPI * n_s * (2.0 - (2.0 + L * ln2) * std::exp2(-L)) / ln2;
    const int K = (int)std::max(-100.0, std::min(100.0, std::floor(30.0 - std::log2(std::max(ts, 1e-300)))));
    P.qinv = std::ldexp(1.0, -K);
    h->qscale = (float)std::ldexp(1.0, K);
    // close-pair correction: pairs nearer than d_c = 0.005 max(1, |s|max / 4) scaled units
    // (the FP32 rounding of |s| moves them most relative to their separation; what it
    // leaves in the farther pairs grows like |s|max / d_c); hashed cells 2.1 d_c wide.
    // d_c is held to half a neighbour per ion at the mean density, 4/3 pi d_c^3 n_s <= 1/2:
    // in domains far longer than the Debye length (|s|max > 10) the rule would put hundreds
    // of ions within d_c of each ion and the walk of its cells would cost more than the
    // pair forces; there the FP32 coordinates bound the per-ion accuracy instead
    const double smax = std::sqrt(Rs * Rs + Hs * Hs);
    const double dc_cap = std::cbrt(0.375 / (kPI * std::max(n_s, 1e-300)));
    const double dc = std::min(0.005 * std::max(1.0, 0.25 * smax), dc_cap);
    P.cp_dc2 = dc * dc;
    P.cp_hinv = (float)(1.0 / (2.1 * dc));
    P.cp_on = !(p->flags & (OD_F_NO_IONION | OD_F_FP64_PAIRS));
    double* o = h->info;
    o[0] = lam;
    o[1] = cs;
    o[2] = P.sig;
    o[3] = P.sig_n;
    o[4] = P.u;
    o[5] = P.E;
    o[6] = P.q;
    o[7] = P.m;
    o[8] = Jb / J;
    o[9] = Jt / J;
    o[10] = Js / J;
    o[11] = (double)P.Tb;
    o[12] = (double)P.Tbt;
    o[13] = (double)P.Tcoll;
}

void set_field_coeffs(Phys& P, const double* alpha, bool on)
{
    for (int t = 0; t < 10; ++t) P.Gc[t] = P.Kc[t] = 0.0;
    P.eout = on ? 1 : 0;
    if (!on) return;
    for (int t = 0; t < 15; ++t) {
        const int a = kPowR[t], b = kPowZ[t];
        if (a >= 1) P.Gc[mono_index(a - 1, b)] += 2.0 * a * alpha[t];
        if (b >= 1) P.Kc[mono_index(a, b - 1)] += 2.0 * b * alpha[t];
    }
}

// App. A: potential of the uniform ion fill on the (r, z) grid, then the 15-term fit
int build_eout(od_handle* h, const od_params* p)
{
    const int nx = p->eout_grid > 0 ? p->eout_grid : 40, nz = nx, nq = 64;
    const double lam = 1.0 / h->P.lam_inv;
    std::vector<double> gx, gw;
    gl_nodes(nq, gx, gw);
    const int nodes = (nx + 1) * (nz + 1);
    double *d_gl = nullptr, *d_out = nullptr;
    OD_CK(h, cudaMalloc(&d_gl, sizeof(double) * 2 * nq));
    OD_CK(h, cudaMalloc(&d_out, sizeof(double) * nodes));
    OD_CK(h, cudaMemcpyAsync(d_gl, gx.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, h->stream));
    OD_CK(h, cudaMemcpyAsync(d_gl + nq, gw.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, h->stream));
    OD_LK(h, launch_eout_grid(p->R, p->H, lam, nx, nz, nq, d_gl, d_gl + nq, d_out, h->stream));
    std::vector<double> I(nodes);
    OD_CK(h, cudaMemcpyAsync(I.data(), d_out, sizeof(double) * nodes, cudaMemcpyDeviceToHost, h->stream));
    OD_CK(h, cudaStreamSynchronize(h->stream));
    cudaFree(d_gl);
    cudaFree(d_out);
    // Phi_ext = Phi_0 - Phi_cyl with Phi_0 = 0; Phi_cyl = Z e n_inf / (4 pi eps0) * I
    const double pref = p->ion_charge_number * kQE * p->n_inf / (4.0 * kPI * kEPS0);
    const double hz = 0.5 * p->H;
    std::vector<double> A((size_t)nodes * 15), b(nodes);
    for (int kr = 0; kr <= nx; ++kr)
        for (int kz = 0; kz <= nz; ++kz) {
            const int row = kr * (nz + 1) + kz;
            const double rho2 = (double)kr * kr / ((double)nx * nx), zeta2 = (double)kz * kz / ((double)nz * nz);
            b[row] = -pref * I[row];
            for (int t = 0; t < 15; ++t) A[(size_t)t * nodes + row] = std::pow(rho2, kPowR[t]) * std::pow(zeta2, kPowZ[t]);
        }
    double beta[15];
    if (!lsq_mgs(nodes, 15, A, b, beta)) return fail(h, OD_EINVAL, "E_out fit is singular");
    for (int t = 0; t < 15; ++t)
        h->alpha[t] = beta[t] / (std::pow(p->R * p->R, kPowR[t]) * std::pow(hz * hz, kPowZ[t]));
    return OD_OK;
}

// balanced partition of the all-pairs work for pair-kernel variant v
ForceArgs plan_forces(int N, int v, int sms, int units_per_block, int bps_cap)
{
    ForceArgs F{};
    const ForceVariant fv = force_variant(v);
    F.TI = fv.BT * fv.IPT;
    F.n_pad = N == 0 ? 0 : (N + F.TI - 1) / F.TI * F.TI;
    if (F.n_pad == 0) return F;
    const int n_it = F.n_pad / F.TI;
    const int occ = force_blocks_per_sm(v);
    const long long gmax = (long long)sms * (bps_cap > 0 ? std::min(bps_cap, occ) : occ);
    if (fv.sym) {
        // tile pairs (I, J >= I) into the fixed-point accumulators; units have a fixed
        // size, so units_per_block is unused
        F.sym = 1;
        F.JC = F.TI;
        F.JS = n_it;
        F.W = 0;
        F.U = (long long)n_it * (n_it + 1) / 2;
        F.G = (int)std::min<long long>(gmax, F.U);
        return F;
    }
    long long js = (units_per_block * gmax + n_it - 1) / n_it;
    js = std::max(1ll, std::min(js, (long long)F.n_pad / fv.BT));
    long long jc = ((F.n_pad + js - 1) / js + fv.BT - 1) / fv.BT * fv.BT;
    F.JC = (int)jc;
    F.JS = (int)((F.n_pad + jc - 1) / jc);
    F.U = (long long)n_it * F.JS;
    F.G = (int)std::min<long long>(gmax, F.U);
    int W = 1;
    for (int t = 0; t < n_it; ++t) {
        const long long u0 = (long long)t * F.JS, u1 = u0 + F.JS - 1;
        const int g0 = (int)(((u0 + 1) * F.G - 1) / F.U), g1 = (int)(((u1 + 1) * F.G - 1) / F.U);
        W = std::max(W, g1 - g0 + 1);
    }
    F.W = W;
    return F;
}

// untuned choice: ordered pairs for small runs (many small units spread over the SMs),
// the packed symmetric kernel (half the pair evaluations) with 512-ion tiles above 32k ions
int default_variant(int N)
{
    if (N <= 4096) return 0;
    if (N <= 32768) return 2;
    return 17;  // k_forces_sym2<64,8>
}

int ensure_part(od_handle* h)
{
    const long long need = (long long)h->F.W * h->F.n_pad;
    if (need == 0) return OD_OK;  // symmetric kernels: fixed-point accumulators only
    if (need <= h->part_cap) return OD_OK;
    if (h->B.part) cudaFree(h->B.part);
    h->B.part = nullptr;
    OD_CK(h, cudaMalloc(&h->B.part, sizeof(float4) * std::max(need, 1ll)));
    h->part_cap = need;
    return OD_OK;
}

// the cutoff's plan: symmetric tiles of 512 z-sorted ions whose sums go to the
// fixed-point accumulators at the ions' sorted positions
ForceArgs plan_cut(const od_handle* h, int N)
{
    ForceArgs F{};
    F.TI = 512;
    F.n_pad = N == 0 ? 0 : (N + F.TI - 1) / F.TI * F.TI;
    const int T = F.n_pad / F.TI;
    F.sym = 1;
    F.cut = 1;
    F.JC = F.TI;
    F.JS = T;
    F.W = 0;
    F.U = (long long)T * (T + 1) / 2;
    F.G = h->cut_grid;
    const double ls = 1.4426950408889634 * h->P.lam_inv;
    F.cut_s0 = (float)(h->r_switch * ls);
    F.cut_inv_w = (float)(1.0 / ((h->r_cut - h->r_switch) * ls));
    F.rank = h->C.rank;
    return F;
}

// the fixed-point accumulators, error word, unit queue and live count of the run
void attach_sums(const od_handle* h, ForceArgs& F)
{
    F.psum = h->B.psum;
    F.psum_ld = h->B.psum_ld;
    F.qscale = h->qscale;
    F.err = (int*)((char*)h->B.ctrl + offsetof(Ctrl, err));
    F.sched = h->d_sched;
    F.n_live = (const int*)((const char*)h->B.ctrl + offsetof(Ctrl, n_cur));
}

int replan(od_handle* h, int N)
{
    h->P.N = N;
    if (h->variant < 0 || h->variant >= num_force_variants()) h->variant = default_variant(N);
    if (h->P.flags & OD_F_FP64_PAIRS) {
        // one partial slot per ion (the FP64 kernel's): an ordered plan of 128-ion tiles
        // whose units are the tiles themselves, so every tile has a single slot
        ForceArgs F{};
        F.TI = 128;
        F.n_pad = N == 0 ? 0 : (N + 1023) / 1024 * 1024;
        F.JC = F.n_pad;
        F.JS = 1;
        F.U = F.n_pad / F.TI;
        F.G = (int)F.U;
        F.W = 1;
        h->F = F;
    } else {
        h->F = h->cut_on ? plan_cut(h, N) : plan_forces(N, h->variant, h->sms, h->upb, h->bps);
    }
    attach_sums(h, h->F);
    h->P.n_pad = h->F.n_pad;
    if (h->F.n_pad > h->npad_cap) return fail(h, OD_EOVERFLOW, "padded ion count exceeds the buffer");
    return ensure_part(h);
}

// the step's pair-force stage: all pairs (the variant's kernel) or the cutoff's chain
int launch_pairs(od_handle* h, int after_push)
{
    if (h->cut_on) return launch_forces_cut(h->P, h->B, h->F, h->C, h->cut_grid, h->stream);
    if (h->P.flags & OD_F_FP64_PAIRS) return launch_forces_f64(h->P, h->B, after_push, h->stream);
    return launch_forces(h->P, h->B, h->F, h->variant, h->stream);
}

// ion count the plans are made for: the live count, or the capacity under the flux rule
int plan_n(const od_handle* h, long long n_live)
{
    return (h->P.flags & OD_F_FLUX_INJECT) ? (int)h->cap : (int)n_live;
}

int read_error_word(od_handle* h)
{
    int err = 0;
    OD_CK(h, cudaMemcpyAsync(&err, (char*)h->B.ctrl + offsetof(Ctrl, err), sizeof(int), cudaMemcpyDeviceToHost,
                             h->stream));
    OD_CK(h, cudaStreamSynchronize(h->stream));
    if (err & ERR_NAN) return fail(h, OD_ENAN, "non-finite ion position or velocity");
    if (err & ERR_TIMEOUT) return fail(h, OD_ETIMEOUT, "device-side wait hit its limit (scan look-back)");
    if (err & ERR_PLACE) return fail(h, OD_EINVAL, "initial ion placement failed (grains fill the domain?)");
    if (err & ERR_OVERFLOW) return fail(h, OD_EOVERFLOW, "ion capacity exceeded");
    if (err & ERR_RANGE)
        return fail(h, OD_ERANGE, "a pair-force partial sum left the fixed-point range (two ions nearly coincide)");
    return OD_OK;
}

// forces for the current state (creation or replaced ions): FP32 positions and
// close-pair lists rebuilt, pair forces, accelerations, Eq. 1 force
int force_eval(od_handle* h)
{
    OD_LK(h, launch_fpos(h->P, h->B, (int)(h->host_step & 1), h->stream));
    OD_LK(h, launch_pairs(h, 0));
    OD_LK(h, launch_kick(h->P, h->B, h->F, 1, h->stream));  // with the grain tail
    return OD_OK;
}

int launch_density(od_handle* h)
{
    if (!h->d_hist) return OD_OK;
    OD_LK(h, launch_hist(h->P, h->B, h->d_hist, h->hist_nr, h->hist_nz, h->hist_nr / h->P.R, h->hist_nz / h->P.H,
                         h->sms, h->stream));
    return OD_OK;
}

// the next step's injection samples on the second stream, beside the pair forces (fork
// after the scan, which fixes their ids; joined by join_ahead before the step ends)
// and this step's collision velocities on a third (joined by join_collide before the kick)
int fork_ahead(od_handle* h)
{
    if (!h->aux) return OD_OK;
    OD_CK(h, cudaEventRecord(h->ev_fork, h->stream));
    OD_CK(h, cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
    OD_LK(h, launch_inject_ahead(h->P, h->B, h->aux));
    OD_CK(h, cudaEventRecord(h->ev_join, h->aux));
    OD_CK(h, cudaStreamWaitEvent(h->aux2, h->ev_fork, 0));
    OD_LK(h, launch_collide_ahead(h->P, h->B, h->aux2));
    OD_CK(h, cudaEventRecord(h->ev_join2, h->aux2));
    return OD_OK;
}

int join_collide(od_handle* h)
{
    if (!h->aux) return OD_OK;
    OD_CK(h, cudaStreamWaitEvent(h->stream, h->ev_join2, 0));
    return OD_OK;
}

int join_ahead(od_handle* h)
{
    if (!h->aux) return OD_OK;
    OD_CK(h, cudaStreamWaitEvent(h->stream, h->ev_join, 0));
    return OD_OK;
}

int launch_step(od_handle* h)
{
    int rc;
    OD_LK(h, launch_push_scan(h->P, h->B, h->stream));
    if ((rc = fork_ahead(h))) return rc;
    OD_LK(h, launch_pairs(h, 1));
    if ((rc = join_collide(h))) return rc;
    OD_LK(h, launch_kick(h->P, h->B, h->F, 0, h->stream));  // with the grain tail
    if ((rc = join_ahead(h))) return rc;
    return launch_density(h);
}

int ensure_series(od_handle* h, long long need)
{
    if (need <= h->series_cap) return OD_OK;
    long long nc = std::max({need, 2 * h->series_cap, 1024ll});
    double* ns = nullptr;
    int* ne = nullptr;
    OD_CK(h, cudaMalloc(&ns, sizeof(double) * nc * MAXD * REC));
    OD_CK(h, cudaMalloc(&ne, sizeof(int) * nc * EV));
    OD_CK(h, cudaMemsetAsync(ns, 0, sizeof(double) * nc * MAXD * REC, h->stream));
    OD_CK(h, cudaMemsetAsync(ne, 0, sizeof(int) * nc * EV, h->stream));
    if (h->series_cap > 0) {
        OD_CK(h, cudaMemcpyAsync(ns, h->d_series, sizeof(double) * h->series_cap * MAXD * REC,
                                 cudaMemcpyDeviceToDevice, h->stream));
        OD_CK(h, cudaMemcpyAsync(ne, h->d_evseries, sizeof(int) * h->series_cap * EV, cudaMemcpyDeviceToDevice,
                                 h->stream));
    }
    struct {
        double* s;
        int* e;
        long long c;
    } ptrs = {ns, ne, nc};
    static_assert(offsetof(Ctrl, evseries) == offsetof(Ctrl, series) + sizeof(double*), "layout");
    static_assert(offsetof(Ctrl, series_cap) == offsetof(Ctrl, evseries) + sizeof(int*), "layout");
    OD_CK(h, cudaMemcpyAsync((char*)h->B.ctrl + offsetof(Ctrl, series), &ptrs, sizeof(ptrs), cudaMemcpyHostToDevice,
                             h->stream));
    OD_CK(h, cudaStreamSynchronize(h->stream));
    if (h->d_series) cudaFree(h->d_series);
    if (h->d_evseries) cudaFree(h->d_evseries);
    h->d_series = ns;
    h->d_evseries = ne;
    h->series_cap = nc;
    return OD_OK;
}

// staging for host arrays crossing the ABI: one device buffer and one pinned host buffer
// of 9 doubles per ion of capacity (x, v, a interleaved) plus the ids
int ensure_io(od_handle* h)
{
    if (h->d_io) return OD_OK;
    OD_CK(h, cudaMalloc(&h->d_io, sizeof(double) * 9 * h->cap));
    OD_CK(h, cudaMallocHost(&h->h_io, sizeof(double) * 9 * h->cap));
    OD_CK(h, cudaMallocHost(&h->h_ioid, sizeof(uint64_t) * h->cap));
    return OD_OK;
}

// host memory the GPU can copy from directly (page-locked or registered)
bool host_pinned(const void* p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost;
}

void free_cut(od_handle* h)
{
    CutBufs& C = h->C;
    void* ptrs[] = {C.bcount, C.boff, C.bsum, C.perm, C.rank, C.fsort, C.box_lo, C.box_hi,
                    C.units, C.n_units, C.ucnt, C.ustart};
    for (void* q : ptrs) cudaFree(q);
    C = CutBufs{};
}

void free_all(od_handle* h)
{
    for (int b = 0; b < 2; ++b) {
        cudaFree(h->B.x[b]);
        cudaFree(h->B.v[b]);
        cudaFree(h->B.id[b]);
    }
    cudaFree(h->B.acc);
    cudaFree(h->B.fpos);
    cudaFree(h->B.part);
    cudaFree(h->B.psum);
    cudaFree(h->B.cp_head);
    cudaFree(h->B.cp_next);
    cudaFree(h->B.tile_status);
    cudaFree(h->B.inj);
    cudaFree(h->B.rem);
    cudaFree(h->B.dpart);
    cudaFree(h->B.ctrl);
    cudaFree(h->d_stats);
    cudaFree(h->d_sched);
    cudaFree(h->d_vtab);
    cudaFree(h->d_series);
    cudaFree(h->d_evseries);
    cudaFree(h->d_hist);
    cudaFree(h->d_io);
    cudaFreeHost(h->h_io);
    cudaFreeHost(h->h_ioid);
    free_cut(h);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    if (h->gexec_k) cudaGraphExecDestroy(h->gexec_k);
    if (h->graph_k) cudaGraphDestroy(h->graph_k);
    for (auto& e : h->ev)
        if (e) cudaEventDestroy(e);
    for (auto& e : h->pev)
        if (e) cudaEventDestroy(e);
    cudaFree(h->B.inj_ahead);
    cudaFree(h->B.coll_v);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->ev_join2) cudaEventDestroy(h->ev_join2);
    if (h->aux) cudaStreamDestroy(h->aux);
    if (h->aux2) cudaStreamDestroy(h->aux2);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

int create_impl(const od_params* p, od_handle* h)
{
    int dev = 0;
    OD_CK(h, cudaGetDevice(&dev));
    OD_CK(h, cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev));
    if (p->cuda_stream) {
        h->stream = (cudaStream_t)p->cuda_stream;
    } else {
        OD_CK(h, cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
        h->own_stream = true;
    }
    h->prm = *p;
    for (int k = 0; k < p->n_dust; ++k) h->prm_dust[k] = p->dust[k];
    h->prm.dust = nullptr;
    h->prm.eout_coeffs = nullptr;
    h->prm.cuda_stream = nullptr;
    derive(p, h->P, h);
    {
        std::vector<double> tab;
        build_vtab(h->P.u, h->P.sig, tab, h->P.gmax_b, h->P.gmax_t);
        OD_CK(h, cudaMalloc(&h->d_vtab, sizeof(double) * tab.size()));
        OD_CK(h, cudaMemcpyAsync(h->d_vtab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, h->stream));
        OD_CK(h, cudaStreamSynchronize(h->stream));
        h->P.vtab = h->d_vtab;
    }
    const bool eout_on = !(p->flags & OD_F_NO_EOUT);
    if (p->eout_coeffs) {
        std::memcpy(h->alpha, p->eout_coeffs, sizeof(double) * 15);
    } else if (eout_on) {
        int rc = build_eout(h, p);
        if (rc) return rc;
    }
    set_field_coeffs(h->P, h->alpha, eout_on);
    const int N = h->P.N;  // initial ions
    // with the flux injection rule N varies: buffers and plans are sized for a capacity
    const bool flux = (p->flags & OD_F_FLUX_INJECT) != 0;
    const int n_plan = flux ? N + std::max(256, (N + 3) / 4) : N;
    h->cap = std::max(n_plan, 1);
    h->npad_cap = ((long long)h->cap + 1023) / 1024 * 1024;
    h->nb_cap = (h->cap + kick_block() - 1) / kick_block();
    // untuned runs start from the size-based default; batch members are re-planned by
    // their batch (ordered-pair units) and need no symmetric partial slots meanwhile
    h->variant = h->batch_member ? 3 : -1;
    Bufs& B = h->B;
    B.cap = h->cap;
    for (int b = 0; b < 2; ++b) {
        OD_CK(h, cudaMalloc(&B.x[b], sizeof(double) * 3 * h->cap));
        OD_CK(h, cudaMalloc(&B.v[b], sizeof(double) * 3 * h->cap));
        OD_CK(h, cudaMalloc(&B.id[b], sizeof(unsigned long long) * h->cap));
    }
    OD_CK(h, cudaMalloc(&B.acc, sizeof(float4) * h->npad_cap));
    OD_CK(h, cudaMalloc(&B.fpos, sizeof(float4) * h->npad_cap));
    // fixed-point pair sums [3][npad_cap] (zero between evaluations) and the close-pair
    // cell buckets (a power of two) and links
    B.psum_ld = h->npad_cap;
    OD_CK(h, cudaMalloc(&B.psum, sizeof(long long) * 3 * h->npad_cap));
    OD_CK(h, cudaMemsetAsync(B.psum, 0, sizeof(long long) * 3 * h->npad_cap, h->stream));
    // (32 buckets per ion up to 2^16 ions and 8 up to 2^18: the walks then meet few ions
    // of other cells; two per ion above, which keeps the grid near the L2's size)
    unsigned long long nbk = 1024;
    const unsigned long long per_ion = h->cap <= (1 << 16) ? 32ull : h->cap <= (1 << 18) ? 8ull : 2ull;
    const unsigned long long want = per_ion * (unsigned long long)h->cap;
    while (nbk < want) nbk <<= 1;
    h->P.cp_mask = (unsigned)(nbk - 1);
    OD_CK(h, cudaMalloc(&B.cp_head, sizeof(unsigned long long) * nbk));
    OD_CK(h, cudaMemsetAsync(B.cp_head, 0, sizeof(unsigned long long) * nbk, h->stream));
    OD_CK(h, cudaMalloc(&B.cp_next, sizeof(int) * h->cap));
    // one status word per scan tile: single runs scan 256-ion tiles, batch members 128
    const long long scan_tile = std::min(push_tile(), BATCH_TILE);
    const long long ntiles = (h->cap + scan_tile - 1) / scan_tile;
    h->scan_tiles_cap = ntiles;
    OD_CK(h, cudaMalloc(&B.tile_status, sizeof(unsigned long long) * ntiles));
    OD_CK(h, cudaMemsetAsync(B.tile_status, 0, sizeof(unsigned long long) * ntiles, h->stream));
    OD_CK(h, cudaMalloc(&B.inj, sizeof(Inj) * h->cap));
    OD_CK(h, cudaMalloc(&B.rem, sizeof(Rem) * h->cap));
    OD_CK(h, cudaMalloc(&B.inj_ahead, sizeof(Inj) * INJ_AHEAD));
    if (!h->batch_member) {
        // single runs draw the next step's injection samples and this step's collision
        // velocities on two more streams, beside the pair forces
        OD_CK(h, cudaMalloc(&B.coll_v, sizeof(double) * 3 * h->cap));
        OD_CK(h, cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking));
        OD_CK(h, cudaStreamCreateWithFlags(&h->aux2, cudaStreamNonBlocking));
        OD_CK(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        OD_CK(h, cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
        OD_CK(h, cudaEventCreateWithFlags(&h->ev_join2, cudaEventDisableTiming));
    }
    OD_CK(h, cudaMalloc(&B.dpart, sizeof(double) * h->nb_cap * MAXD * 3));
    OD_CK(h, cudaMalloc(&B.ctrl, sizeof(Ctrl)));
    OD_CK(h, cudaMalloc(&h->d_stats, sizeof(double) * 2 * MAXD * REC));
    OD_CK(h, cudaMalloc(&h->d_sched, 2 * sizeof(unsigned long long)));
    OD_CK(h, cudaMemsetAsync(h->d_sched, 0, 2 * sizeof(unsigned long long), h->stream));
    Ctrl c0;
    std::memset(&c0, 0, sizeof(c0));
    c0.next_id = (unsigned long long)N;
    c0.n_cur = N;
    c0.cp_epoch = 1;  // bucket words start at epoch 0, which no build uses
    for (int k = 0; k < p->n_dust; ++k) c0.Q[k] = p->charge_model == OD_Q_OML ? 0.0 : p->dust[k].q0;
    OD_CK(h, cudaMemcpyAsync(B.ctrl, &c0, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream));
    OD_LK(h, launch_grain_eout(h->P, B, h->stream));
    if (p->charge_model == OD_Q_OML && p->n_dust > 0) {
        // the grains' OML floating charges, solved on the device
        std::vector<double> gx, gw;
        gl_nodes(96, gx, gw);
        double* d_gl = nullptr;
        OD_CK(h, cudaMalloc(&d_gl, sizeof(double) * 2 * gx.size()));
        OD_CK(h, cudaMemcpyAsync(d_gl, gx.data(), sizeof(double) * gx.size(), cudaMemcpyHostToDevice, h->stream));
        OD_CK(h, cudaMemcpyAsync(d_gl + gx.size(), gw.data(), sizeof(double) * gw.size(), cudaMemcpyHostToDevice,
                                 h->stream));
        const int lrc = launch_oml_charge(h->P, B, p->n_inf, p->ion_mass, p->ion_charge_number, p->T_e, (int)gx.size(),
                                          d_gl, d_gl + gx.size(), h->stream);
        const cudaError_t se = cudaStreamSynchronize(h->stream);
        cudaFree(d_gl);
        if (lrc) return cuda_fail(h, (cudaError_t)lrc, "launch_oml_charge");
        OD_CK(h, se);
    }
    int rc = replan(h, n_plan);
    if (rc) return rc;
    Phys Pi = h->P;
    Pi.N = N;  // the initial ions only
    OD_LK(h, launch_init_ions(Pi, B, h->stream));
    OD_LK(h, launch_fpos(h->P, B, 0, h->stream));
    rc = force_eval(h);
    if (rc) return rc;
    rc = ensure_series(h, 1024);
    if (rc) return rc;
    for (auto& e : h->ev) OD_CK(h, cudaEventCreate(&e));
    return read_error_word(h);
}

}  // namespace host
}  // namespace od

extern "C" {

int od_create(const od_params* p, od_handle** out)
{
    if (!out) return fail(nullptr, OD_EINVAL, "out is NULL");
    *out = nullptr;
    std::string msg;
    int rc = validate(p, msg);
    if (rc) return fail(nullptr, rc, msg);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(nullptr, OD_ENODEV, "no CUDA device");
    od_handle* h = new od_handle();
    rc = create_impl(p, h);
    if (rc) {
        g_create_error = h->err;
        free_all(h);
        delete h;
        return rc;
    }
    *out = h;
    return OD_OK;
}

// per-kernel times of the steps recorded in the profiling ring (waits for the last one)
int drain_profile(od_handle* h)
{
    OD_CK(h, cudaEventSynchronize(h->pev[5 * h->pev_used - 1]));
    for (int s = 0; s < h->pev_used; ++s)
        for (int k = 0; k < 4; ++k) {
            float ms = 0.f;
            OD_CK(h, cudaEventElapsedTime(&ms, h->pev[5 * s + k], h->pev[5 * s + k + 1]));
            h->kms[k] += ms;
            h->klaunch[k] += 1;
        }
    h->pev_used = 0;
    return OD_OK;
}

int od_step(od_handle* h, int64_t n)
{
    if (!h || n < 0) return fail(h, OD_EINVAL, "bad handle or step count");
    if (h->batch_member) return fail(h, OD_EINVAL, "this run belongs to a batch: step it with od_batch_step");
    if (n == 0) return OD_OK;
    int rc = ensure_series(h, h->host_step + n);
    if (rc) return rc;
    const bool direct = h->profiling || (h->P.flags & OD_F_NO_GRAPH);
    // one step per graph, and STEP_GRAPH_K steps per graph for long calls: a small run's
    // step is a few tens of microseconds, of which a graph launch per step would be a
    // good part
    auto capture = [h](int steps, cudaGraph_t* graph, cudaGraphExec_t* exec) -> int {
        if (*exec) cudaGraphExecDestroy(*exec);
        if (*graph) cudaGraphDestroy(*graph);
        *exec = nullptr;
        *graph = nullptr;
        OD_CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        int lrc = 0;
        for (int k = 0; k < steps && !lrc; ++k) lrc = launch_step(h);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->stream, &g);
        if (lrc) {
            if (g) cudaGraphDestroy(g);
            return lrc;
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
        *graph = g;
        OD_CK(h, cudaGraphInstantiate(exec, g, 0));
        return OD_OK;
    };
    if (!direct && !h->graph_ok) {
        h->graph_k_ok = false;
        if ((rc = capture(1, &h->graph, &h->gexec))) return rc;
        h->graph_ok = true;
    }
    if (!direct && n >= STEP_GRAPH_K && !h->graph_k_ok) {
        if ((rc = capture(STEP_GRAPH_K, &h->graph_k, &h->gexec_k))) return rc;
        h->graph_k_ok = true;
    }
    for (int64_t s = 0; s < n; ++s) {
        if (!direct && n - s >= STEP_GRAPH_K) {
            OD_CK(h, cudaGraphLaunch(h->gexec_k, h->stream));
            s += STEP_GRAPH_K - 1;
            continue;
        }
        if (direct) {
            if (h->profiling) {
                // events around each kernel, read PROF_RING steps at a time, so that the
                // host runs ahead of the device and leaves no gap between steps
                cudaEvent_t* e = &h->pev[5 * h->pev_used];
                OD_CK(h, cudaEventRecord(e[0], h->stream));
                OD_LK(h, launch_push_scan(h->P, h->B, h->stream));
                OD_CK(h, cudaEventRecord(e[1], h->stream));
                if ((rc = fork_ahead(h))) return rc;
                OD_LK(h, launch_pairs(h, 1));
                OD_CK(h, cudaEventRecord(e[2], h->stream));
                if ((rc = join_collide(h))) return rc;
                OD_LK(h, launch_kick(h->P, h->B, h->F, 0, h->stream));  // with the grain tail
                OD_CK(h, cudaEventRecord(e[3], h->stream));
                OD_CK(h, cudaEventRecord(e[4], h->stream));
                if ((rc = join_ahead(h))) return rc;
                if ((rc = launch_density(h))) return rc;
                if (++h->pev_used == PROF_RING && (rc = drain_profile(h))) return rc;
            } else {
                rc = launch_step(h);
                if (rc) return rc;
            }
        } else {
            OD_CK(h, cudaGraphLaunch(h->gexec, h->stream));
        }
    }
    if (h->profiling && h->pev_used && (rc = drain_profile(h))) return rc;
    h->host_step += n;
    if (h->d_hist) h->hist_samples += n;
    return read_error_word(h);
}

void od_destroy(od_handle* h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

int od_dust_terms(od_handle* h, double* mean, double* se)
{
    if (!h) return fail(h, OD_EINVAL, "bad handle");
    OD_LK(h, launch_stats(h->P, h->B, h->d_stats, h->stream));
    double buf[2 * MAXD * REC];
    OD_CK(h, cudaMemcpyAsync(buf, h->d_stats, sizeof(buf), cudaMemcpyDeviceToHost, h->stream));
    OD_CK(h, cudaStreamSynchronize(h->stream));
    const int n = h->P.D * REC;
    if (mean) std::memcpy(mean, buf, sizeof(double) * n);
    if (se) std::memcpy(se, buf + MAXD * REC, sizeof(double) * n);
    return OD_OK;
}

int od_dust_state(od_handle* h, double* q, double* F)
{
    double mean[MAXD * REC];
    int rc = od_dust_terms(h, mean, nullptr);
    if (rc) return rc;
    for (int k = 0; k < h->P.D; ++k) {
        const double* r = mean + k * REC;
        if (q) q[k] = r[0];
        if (F)
            for (int c = 0; c < 3; ++c) F[3 * k + c] = r[1 + c] + r[4 + c] + r[7 + c] + r[10 + c];
    }
    return OD_OK;
}

int od_series(od_handle* h, int64_t first, int64_t count, double* rec, int32_t* ev)
{
    if (!h) return fail(h, OD_EINVAL, "bad handle");
    if (first < 1 || count < 0 || first + count - 1 > h->host_step || first + count - 1 > h->series_cap)
        return fail(h, OD_EINVAL, "series range outside the steps taken");
    if (count == 0) return OD_OK;
    const int D = h->P.D;
    if (rec) {
        std::vector<double> tmp((size_t)count * MAXD * REC);
        OD_CK(h, cudaMemcpyAsync(tmp.data(), h->d_series + (first - 1) * MAXD * REC, sizeof(double) * tmp.size(),
                                 cudaMemcpyDeviceToHost, h->stream));
        OD_CK(h, cudaStreamSynchronize(h->stream));
        for (int64_t t = 0; t < count; ++t)
            std::memcpy(rec + (t * D) * REC, tmp.data() + t * MAXD * REC, sizeof(double) * D * REC);
    }
    if (ev) {
        OD_CK(h, cudaMemcpyAsync(ev, h->d_evseries + (first - 1) * EV, sizeof(int) * count * EV,
                                 cudaMemcpyDeviceToHost, h->stream));
        OD_CK(h, cudaStreamSynchronize(h->stream));
    }
    return OD_OK;
}

int od_counters(od_handle* h, int64_t* out)
{
    if (!h || !out) return fail(h, OD_EINVAL, "bad argument");
    int n_live = 0;
    OD_CK(h, cudaMemcpyAsync(out, (char*)h->B.ctrl + offsetof(Ctrl, counters), sizeof(long long) * OD_NCOUNT,
                             cudaMemcpyDeviceToHost, h->stream));
    OD_CK(h, cudaMemcpyAsync(&n_live, (char*)h->B.ctrl + offsetof(Ctrl, n_cur), sizeof(int), cudaMemcpyDeviceToHost,
                             h->stream));
    OD_CK(h, cudaStreamSynchronize(h->stream));
    out[13] = h->host_step;
    out[14] = n_live;  // ions alive now (varies under the flux rule)
    return OD_OK;
}

int od_dust_now(od_handle* h, double* q, double* f_orbit)
{
    if (!h) return fail(h, OD_EINVAL, "bad handle");
    Ctrl c;
    OD_CK(h, cudaMemcpyAsync(&c, h->B.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
    OD_CK(h, cudaStreamSynchronize(h->stream));
    for (int k = 0; k < h->P.D; ++k) {
        if (q) q[k] = c.Q[k];
        if (f_orbit)
            for (int j = 0; j < 3; ++j) f_orbit[3 * k + j] = c.f_orbit[k][j];
    }
    return OD_OK;
}

int64_t od_get_ions(od_handle* h, double* x, double* v, double* a, uint64_t* id, int64_t cap)
{
    if (!h) return fail(h, OD_EINVAL, "bad handle");
    int n_live = 0;  // ions alive (it varies under the flux rule)
    OD_CK(h, cudaMemcpyAsync(&n_live, (char*)h->B.ctrl + offsetof(Ctrl, n_cur), sizeof(int), cudaMemcpyDeviceToHost,
                             h->stream));
    OD_CK(h, cudaStreamSynchronize(h->stream));
    const long long N = n_live;
    if ((x || v || a || id) && cap < N) return fail(h, OD_EINVAL, "host arrays too small");
    if (N == 0 || !(x || v || a || id)) return N;
    int rc;
    if ((rc = ensure_io(h))) return rc;
    const int buf = (int)(h->host_step & 1);
    const size_t bytes = sizeof(double) * 3 * N;
    double* const outs[3] = {x, v, a};
    bool staged[3] = {false, false, false};
    for (int k = 0; k < 3; ++k) {
        if (!outs[k]) continue;
        double* dst = h->d_io + 3 * h->cap * k;
        if (k < 2) OD_LK(h, launch_layout(1, k == 0 ? h->B.x[buf] : h->B.v[buf], dst, (int)N, h->cap, h->stream));
        else OD_LK(h, launch_layout(2, h->B.acc, dst, (int)N, h->cap, h->stream));
        staged[k] = !host_pinned(outs[k]);
        OD_CK(h, cudaMemcpyAsync(staged[k] ? h->h_io + 3 * h->cap * k : outs[k], dst, bytes, cudaMemcpyDeviceToHost,
                                 h->stream));
    }
    const bool id_staged = id && !host_pinned(id);
    if (id)
        OD_CK(h, cudaMemcpyAsync(id_staged ? h->h_ioid : id, h->B.id[buf], sizeof(uint64_t) * N,
                                 cudaMemcpyDeviceToHost, h->stream));
    OD_CK(h, cudaStreamSynchronize(h->stream));
    for (int k = 0; k < 3; ++k)
        if (staged[k]) std::memcpy(outs[k], h->h_io + 3 * h->cap * k, bytes);
    if (id_staged) std::memcpy(id, h->h_ioid, sizeof(uint64_t) * N);
    return N;
}

int od_set_ions(od_handle* h, const double* x, const double* v, const double* a, const uint64_t* id, int64_t n,
                uint64_t next_id)
{
    if (!h || n < 0 || (n > 0 && (!x || !v || !id))) return fail(h, OD_EINVAL, "bad argument");
    if (h->batch_member) return fail(h, OD_EINVAL, "the ions of a batch member cannot be replaced");
    if (n > h->cap) return fail(h, OD_EOVERFLOW, "more ions than the handle's capacity");
    const int buf = (int)(h->host_step & 1);
    int rc;
    if (n > 0) {
        if ((rc = ensure_io(h))) return rc;
        const size_t bytes = sizeof(double) * 3 * n;
        const double* const ins[3] = {x, v, a};
        for (int k = 0; k < 3; ++k) {
            if (!ins[k]) continue;
            double* dst = h->d_io + 3 * h->cap * k;
            const double* src = ins[k];
            if (!host_pinned(src)) {
                std::memcpy(h->h_io + 3 * h->cap * k, src, bytes);
                src = h->h_io + 3 * h->cap * k;
            }
            OD_CK(h, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->stream));
            if (k < 2) OD_LK(h, launch_layout(0, dst, k == 0 ? h->B.x[buf] : h->B.v[buf], (int)n, h->cap, h->stream));
            else OD_LK(h, launch_layout(3, dst, h->B.acc, (int)n, h->cap, h->stream));
        }
        const uint64_t* ids = id;
        if (!host_pinned(id)) {
            std::memcpy(h->h_ioid, id, sizeof(uint64_t) * n);
            ids = h->h_ioid;
        }
        OD_CK(h, cudaMemcpyAsync(h->B.id[buf], ids, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, h->stream));
    }
    unsigned long long nid = next_id;
    OD_CK(h, cudaMemcpyAsync((char*)h->B.ctrl + offsetof(Ctrl, next_id), &nid, sizeof(nid), cudaMemcpyHostToDevice,
                             h->stream));
    const int n_live = (int)n;
    OD_CK(h, cudaMemcpyAsync((char*)h->B.ctrl + offsetof(Ctrl, n_cur), &n_live, sizeof(int), cudaMemcpyHostToDevice,
                             h->stream));
    OD_CK(h, cudaStreamSynchronize(h->stream));  // n_live is a host local
    // the step graph holds the plan by value and the plan is a function of the planned
    // ion count: keep it when that is unchanged
    const int n_plan_old = h->P.N;
    if ((rc = replan(h, plan_n(h, n)))) return rc;
    if (h->P.N != n_plan_old) h->graph_ok = false;
    // given accelerations were converted on the device above (the positions and their
    // close-pair lists are refreshed); otherwise evaluate them
    if (a) OD_LK(h, launch_fpos(h->P, h->B, buf, h->stream));
    else if ((rc = force_eval(h))) return rc;
    return read_error_word(h);
}

int od_info(od_handle* h, double* out)
{
    if (!h || !out) return fail(h, OD_EINVAL, "bad argument");
    for (int i = 0; i < 32; ++i) out[i] = h->info[i];
    out[14] = h->P.N;
    for (int t = 0; t < 15; ++t) out[15 + t] = h->alpha[t];
    out[30] = (double)h->cap;
    out[31] = h->sms;
    return OD_OK;
}

int od_set_profiling(od_handle* h, int on)
{
    if (!h) return fail(h, OD_EINVAL, "bad handle");
    if (on && h->pev.empty()) {
        h->pev.assign(5 * PROF_RING, nullptr);
        for (auto& e : h->pev) OD_CK(h, cudaEventCreate(&e));
    }
    h->pev_used = 0;
    h->profiling = on != 0;
    for (int k = 0; k < 4; ++k) {
        h->kms[k] = 0.0;
        h->klaunch[k] = 0;
    }
    return OD_OK;
}

int od_kernel_times(od_handle* h, double* ms, int64_t* launches)
{
    if (!h) return fail(h, OD_EINVAL, "bad handle");
    for (int k = 0; k < 4; ++k) {
        if (ms) ms[k] = h->kms[k];
        if (launches) launches[k] = h->klaunch[k];
    }
    return OD_OK;
}

const char* od_last_error(const od_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int od_oml_charge(const od_params* p, double radius, double* Q)
{
    std::string msg;
    if (!Q || !(radius > 0) || !std::isfinite(radius)) return fail(nullptr, OD_EINVAL, "bad radius or output");
    od_params q = *p;
    q.n_dust = 0;
    const int rc = validate(&q, msg);
    if (rc) return fail(nullptr, rc, msg);
    *Q = oml_charge(p, radius);
    return OD_OK;
}

int od_selftest_wait_timeout(od_handle* h, int64_t polls)
{
    if (!h || polls < 1) return fail(h, OD_EINVAL, "bad handle or poll limit");
    if (h->P.N <= push_tile()) return fail(h, OD_EINVAL, "the wait self-test needs more than one scan tile");
    Phys P = h->P;
    P.spin_limit = polls;
    P.test_hold_tile0 = 1;
    OD_LK(h, launch_push_scan(P, h->B, h->stream));
    OD_LK(h, launch_cp_bump(h->B, h->stream));  // no later build reuses the epoch of the scan's lists
    OD_CK(h, cudaStreamSynchronize(h->stream));
    h->graph_ok = false;
    return read_error_word(h);
}

int od_num_dust(od_handle* h) { return h ? h->P.D : fail(h, OD_EINVAL, "bad handle"); }


}  // extern "C"
