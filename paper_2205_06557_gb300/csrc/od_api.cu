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

#include "od_internal.h"

using namespace od;

namespace {

// CODATA 2018
constexpr double kQE = 1.602176634e-19;
constexpr double kKB = 1.380649e-23;
constexpr double kEPS0 = 8.8541878128e-12;
constexpr double kME = 9.1093837015e-31;
constexpr double kPI = 3.141592653589793238;
constexpr double kTWO32 = 4294967296.0;

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

}  // namespace

void od::set_global_error(const std::string& msg) { g_create_error = msg; }

struct od_handle {
    Phys P{};
    Bufs B{};
    ForceArgs F{};
    int variant = 0;
    int upb = 8;  // pair-kernel work units per persistent block
    int bps = 0;  // persistent pair-kernel CTAs per SM (0 = occupancy limit)
    bool batch_member = false;  // stepped only through its batch (od_batch_step)
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool graph_ok = false;
    long long cap = 0;       // ion capacity
    long long npad_cap = 0;  // fpos capacity
    long long part_cap = 0;  // partial-sum capacity (float4)
    long long nb_cap = 0;    // kick blocks capacity
    long long host_step = 0;
    long long series_cap = 0;
    int sms = 0;
    double alpha[15] = {0};
    double info[32] = {0};
    std::string err;
    bool profiling = false;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    double kms[4] = {0, 0, 0, 0};
    long long klaunch[4] = {0, 0, 0, 0};
    double* d_stats = nullptr;
    double* d_vtab = nullptr;
    double* d_series = nullptr;
    int* d_evseries = nullptr;
    od_params prm{};                     // creation parameters (pointers cleared): checkpoints
    od_dust prm_dust[OD_MAX_DUST] = {};
    unsigned long long* d_hist = nullptr;  // n(r, z) counts [nz][nr] while enabled
    int hist_nr = 0, hist_nz = 0;
    long long hist_samples = 0;
    double* d_io = nullptr;   // device staging of host arrays: x, v, a as [cap][3] each
    double* h_io = nullptr;   // pinned staging for pageable host arrays (same layout)
    uint64_t* h_ioid = nullptr;
    bool cut_on = false;                   // ion-ion cutoff (od_set_cutoff)
    double r_cut = 0.0, r_switch = 0.0;
    CutBufs C{};
    int cut_grid = 1;
};

namespace {

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

#define OD_CK(h, call)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

#define OD_LK(h, call)                                                       \
    do {                                                                     \
        int e_ = (call);                                                     \
        if (e_ != 0) return cuda_fail(h, (cudaError_t)e_, #call);            \
    } while (0)

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
    const int nx = p->eout_grid > 0 ? p->eout_grid : 40, nz = nx, nq = 48;
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
        // tile pairs (I, J >= I); units have a fixed size, so units_per_block is unused
        F.sym = 1;
        F.JC = F.TI;
        F.JS = n_it;
        F.W = n_it;
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
// the packed symmetric kernel with 1024-ion tiles (half the pair evaluations; fastest at
// 200k ions) above 32k ions while its partial slots (N_pad^2 / 1024 x 16 bytes) stay
// within 16 GB, i.e. up to ~1.05 million ions
int default_variant(int N)
{
    if (N <= 4096) return 0;
    if (N <= 32768) return 2;
    const int sym2_1024 = 15;  // k_forces_sym2<256,4>
    const double n = (double)N + 1024.0;
    if (n * n / 1024.0 * 16.0 <= 16.0 * (1ull << 30)) return sym2_1024;
    return 3;
}

int ensure_part(od_handle* h)
{
    const long long need = (long long)h->F.W * h->F.n_pad;
    if (need <= h->part_cap) return OD_OK;
    if (h->B.part) cudaFree(h->B.part);
    h->B.part = nullptr;
    OD_CK(h, cudaMalloc(&h->B.part, sizeof(float4) * std::max(need, 1ll)));
    h->part_cap = need;
    return OD_OK;
}

// the cutoff's plan: symmetric tiles of 512 z-sorted ions, one slot per tile for every
// ion (only the neighbouring tiles' slots are written and read)
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
    F.W = h->C.max_deg;
    F.U = (long long)T * (T + 1) / 2;
    F.G = h->cut_grid;
    const double ls = 1.4426950408889634 * h->P.lam_inv;
    F.cut_s0 = (float)(h->r_switch * ls);
    F.cut_inv_w = (float)(1.0 / ((h->r_cut - h->r_switch) * ls));
    F.nbr_start = h->C.nbr_start;
    F.rank = h->C.rank;
    return F;
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
    if (err & ERR_CUTCAP)
        return fail(h, OD_EOVERFLOW, "cutoff: a tile has more neighbour tiles than its partial slots (the ion "
                                     "density became very uneven); set the cutoff again to resize");
    return OD_OK;
}

// forces for the current state (creation or replaced ions)
int force_eval(od_handle* h)
{
    OD_LK(h, launch_pairs(h, 0));
    OD_LK(h, launch_kick(h->P, h->B, h->F, 1, h->stream));
    OD_LK(h, launch_dust(h->P, h->B, 1, h->stream));
    return OD_OK;
}

int launch_density(od_handle* h)
{
    if (!h->d_hist) return OD_OK;
    OD_LK(h, launch_hist(h->P, h->B, h->d_hist, h->hist_nr, h->hist_nz, h->hist_nr / h->P.R, h->hist_nz / h->P.H,
                         h->sms, h->stream));
    return OD_OK;
}

int launch_step(od_handle* h)
{
    OD_LK(h, launch_push_scan(h->P, h->B, h->stream));
    OD_LK(h, launch_pairs(h, 1));
    OD_LK(h, launch_kick(h->P, h->B, h->F, 0, h->stream));
    OD_LK(h, launch_dust(h->P, h->B, 0, h->stream));
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
    void* ptrs[] = {C.bcount, C.boff, C.bsum, C.perm, C.rank, C.fsort, C.box_lo, C.box_hi, C.nbr_start,
                    C.nbr, C.units, C.n_units, C.cnt, C.ucnt, C.ustart, C.over};
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
    cudaFree(h->B.tile_status);
    cudaFree(h->B.inj);
    cudaFree(h->B.rem);
    cudaFree(h->B.dpart);
    cudaFree(h->B.ctrl);
    cudaFree(h->d_stats);
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
    for (auto& e : h->ev)
        if (e) cudaEventDestroy(e);
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
    const long long ntiles = (h->cap + push_tile() - 1) / push_tile();
    OD_CK(h, cudaMalloc(&B.tile_status, sizeof(unsigned long long) * ntiles));
    OD_CK(h, cudaMemsetAsync(B.tile_status, 0, sizeof(unsigned long long) * ntiles, h->stream));
    OD_CK(h, cudaMalloc(&B.inj, sizeof(Inj) * h->cap));
    OD_CK(h, cudaMalloc(&B.rem, sizeof(Rem) * h->cap));
    OD_CK(h, cudaMalloc(&B.dpart, sizeof(double) * h->nb_cap * MAXD * 3));
    OD_CK(h, cudaMalloc(&B.ctrl, sizeof(Ctrl)));
    OD_CK(h, cudaMalloc(&h->d_stats, sizeof(double) * 2 * MAXD * REC));
    Ctrl c0;
    std::memset(&c0, 0, sizeof(c0));
    c0.next_id = (unsigned long long)N;
    c0.n_cur = N;
    for (int k = 0; k < p->n_dust; ++k)
        c0.Q[k] = p->charge_model == OD_Q_OML ? oml_charge(p, p->dust[k].radius) : p->dust[k].q0;
    OD_CK(h, cudaMemcpyAsync(B.ctrl, &c0, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream));
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

}  // namespace

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

int od_step(od_handle* h, int64_t n)
{
    if (!h || n < 0) return fail(h, OD_EINVAL, "bad handle or step count");
    if (h->batch_member) return fail(h, OD_EINVAL, "this run belongs to a batch: step it with od_batch_step");
    if (n == 0) return OD_OK;
    int rc = ensure_series(h, h->host_step + n);
    if (rc) return rc;
    const bool direct = h->profiling || (h->P.flags & OD_F_NO_GRAPH);
    if (!direct && !h->graph_ok) {
        if (h->gexec) cudaGraphExecDestroy(h->gexec);
        if (h->graph) cudaGraphDestroy(h->graph);
        h->gexec = nullptr;
        h->graph = nullptr;
        OD_CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        int lrc = launch_step(h);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->stream, &g);
        if (lrc) return lrc;
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
        h->graph = g;
        OD_CK(h, cudaGraphInstantiate(&h->gexec, g, 0));
        h->graph_ok = true;
    }
    for (int64_t s = 0; s < n; ++s) {
        if (direct) {
            if (h->profiling) {
                OD_CK(h, cudaEventRecord(h->ev[0], h->stream));
                OD_LK(h, launch_push_scan(h->P, h->B, h->stream));
                OD_CK(h, cudaEventRecord(h->ev[1], h->stream));
                OD_LK(h, launch_pairs(h, 1));
                OD_CK(h, cudaEventRecord(h->ev[2], h->stream));
                OD_LK(h, launch_kick(h->P, h->B, h->F, 0, h->stream));
                OD_CK(h, cudaEventRecord(h->ev[3], h->stream));
                OD_LK(h, launch_dust(h->P, h->B, 0, h->stream));
                OD_CK(h, cudaEventRecord(h->ev[4], h->stream));
                if ((rc = launch_density(h))) return rc;
                OD_CK(h, cudaEventSynchronize(h->ev[4]));
                for (int k = 0; k < 4; ++k) {
                    float ms = 0.f;
                    OD_CK(h, cudaEventElapsedTime(&ms, h->ev[k], h->ev[k + 1]));
                    h->kms[k] += ms;
                    h->klaunch[k] += 1;
                }
            } else {
                rc = launch_step(h);
                if (rc) return rc;
            }
        } else {
            OD_CK(h, cudaGraphLaunch(h->gexec, h->stream));
        }
    }
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
    if ((rc = replan(h, plan_n(h, n)))) return rc;
    h->graph_ok = false;
    OD_LK(h, launch_fpos(h->P, h->B, buf, h->stream));
    // given accelerations were converted on the device above; otherwise evaluate them
    if (!a && (rc = force_eval(h))) return rc;
    return read_error_word(h);
}

int od_set_cutoff(od_handle* h, double r_cut, double r_switch)
{
    if (!h) return fail(h, OD_EINVAL, "bad handle");
    if (h->batch_member) return fail(h, OD_EINVAL, "the cutoff is set on single runs, not batch members");
    if (h->P.flags & OD_F_FLUX_INJECT) return fail(h, OD_EINVAL, "the cutoff needs a fixed ion count (no flux rule)");
    if (h->P.flags & OD_F_FP64_PAIRS) return fail(h, OD_EINVAL, "the cutoff runs on the FP32 kernels only");
    if (!std::isfinite(r_cut) || !std::isfinite(r_switch)) return fail(h, OD_EINVAL, "cutoff: non-finite distance");
    OD_CK(h, cudaStreamSynchronize(h->stream));
    int rc;
    const int buf = (int)(h->host_step & 1);
    if (r_cut <= 0.0) {
        if (!h->cut_on) return OD_OK;
        h->cut_on = false;
        h->r_cut = h->r_switch = 0.0;
        free_cut(h);
        if ((rc = replan(h, h->P.N))) return rc;
        h->graph_ok = false;
        OD_LK(h, launch_fpos(h->P, h->B, buf, h->stream));
        if ((rc = force_eval(h))) return rc;
        OD_CK(h, cudaStreamSynchronize(h->stream));
        return read_error_word(h);
    }
    if (!(r_switch >= 0.0 && r_switch < r_cut)) return fail(h, OD_EINVAL, "cutoff: need 0 <= r_switch < r_cut");
    constexpr int TI = 512;
    const long long npad_max = (h->cap + TI - 1) / TI * TI;
    const int T = (int)(npad_max / TI);
    if (T > CUT_MAX_TILES)
        return fail(h, OD_EINVAL, "cutoff: at most " + std::to_string(CUT_MAX_TILES * TI) + " ions");
    // slabs of about an eighth of the cutoff (the slab-by-warp count matrix stays below
    // 64M entries)
    const long long nblk = (h->cap + 31) / 32;
    int nslab = (int)std::min(65536.0, std::max(1.0, std::ceil(h->P.H / (r_cut / 8.0))));
    while ((long long)nslab * nblk > (64ll << 20) && nslab > 1) nslab = (nslab + 1) / 2;
    const double w = h->P.H / nslab;
    // slot capacity: the tiles within the cutoff plus two tile extents, for a uniform
    // density, with a margin of half again
    const double ext = 2.0 * std::max(w, h->P.H * TI / std::max(1.0, (double)h->P.N));
    const double deg = T * std::min(1.0, (2.0 * r_cut + 2.0 * ext) / h->P.H) + 3.0;
    const int max_deg = (int)std::min<double>(T, std::ceil(1.5 * deg) + 8.0);
    const double slot_bytes = (double)max_deg * npad_max * sizeof(float4);
    if (slot_bytes > 48e9)
        return fail(h, OD_EINVAL, "cutoff: the partial slots would need " + std::to_string(slot_bytes / 1e9) +
                                      " GB (cutoff too long for this domain)");
    free_cut(h);
    CutBufs& C = h->C;
    const double ls = 1.4426950408889634 * h->P.lam_inv;
    C.nslab = nslab;
    C.zoff = (float)(0.5 * h->P.H * ls);
    C.inv_w = (float)(1.0 / (w * ls));
    const double rcs = r_cut * ls * (1.0 + 1e-5);  // box test: never drop a pair inside the cutoff
    C.rc2_tile = (float)(rcs * rcs);
    const double rss = r_switch * ls * (1.0 - 1e-5);  // plain units: never skip a switched pair
    C.rs2_tile = (float)(rss * rss);
    C.max_deg = max_deg;
    C.err = (int*)((char*)h->B.ctrl + offsetof(Ctrl, err));
    const long long M = (long long)nslab * nblk;
    const long long nchunk = (M + 8191) / 8192;
    OD_CK(h, cudaMalloc(&C.bcount, sizeof(int) * M));
    OD_CK(h, cudaMalloc(&C.boff, sizeof(int) * M));
    OD_CK(h, cudaMalloc(&C.bsum, sizeof(int) * nchunk));
    OD_CK(h, cudaMalloc(&C.perm, sizeof(int) * h->cap));
    OD_CK(h, cudaMalloc(&C.rank, sizeof(int) * h->cap));
    OD_CK(h, cudaMalloc(&C.fsort, sizeof(float4) * npad_max));
    OD_CK(h, cudaMalloc(&C.box_lo, sizeof(float4) * T));
    OD_CK(h, cudaMalloc(&C.box_hi, sizeof(float4) * T));
    OD_CK(h, cudaMalloc(&C.nbr_start, sizeof(int) * (T + 1)));
    OD_CK(h, cudaMalloc(&C.nbr, sizeof(int) * (size_t)T * T));
    OD_CK(h, cudaMalloc(&C.units, sizeof(int4) * ((size_t)T * (T + 1) / 2)));
    OD_CK(h, cudaMalloc(&C.n_units, sizeof(int)));
    OD_CK(h, cudaMalloc(&C.cnt, sizeof(int) * T));
    OD_CK(h, cudaMalloc(&C.ucnt, sizeof(int) * T));
    OD_CK(h, cudaMalloc(&C.ustart, sizeof(int) * T));
    OD_CK(h, cudaMalloc(&C.over, sizeof(int)));
    h->cut_on = true;
    h->r_cut = r_cut;
    h->r_switch = r_switch;
    h->cut_grid = h->sms * cut_blocks_per_sm(2);
    if ((rc = replan(h, h->P.N))) return rc;
    OD_LK(h, launch_cut_dummies(C, h->P.N, h->F.n_pad, h->stream));
    OD_LK(h, launch_fpos(h->P, h->B, buf, h->stream));
    h->graph_ok = false;
    if ((rc = force_eval(h))) return rc;
    OD_CK(h, cudaStreamSynchronize(h->stream));
    return read_error_word(h);
}

int od_density_enable(od_handle* h, int32_t nr, int32_t nz)
{
    if (!h || nr < 0 || nz < 0 || nr > 4096 || nz > 4096 || (long long)nr * nz > (1ll << 22) || ((nr == 0) != (nz == 0)))
        return fail(h, OD_EINVAL, "bad density map size");
    if (h->batch_member) return fail(h, OD_EINVAL, "density maps are kept for single runs, not batch members");
    OD_CK(h, cudaStreamSynchronize(h->stream));
    cudaFree(h->d_hist);
    h->d_hist = nullptr;
    h->hist_nr = nr;
    h->hist_nz = nz;
    h->hist_samples = 0;
    h->graph_ok = false;
    if (nr == 0) return OD_OK;
    OD_CK(h, cudaMalloc(&h->d_hist, sizeof(unsigned long long) * nr * nz));
    OD_CK(h, cudaMemsetAsync(h->d_hist, 0, sizeof(unsigned long long) * nr * nz, h->stream));
    OD_CK(h, cudaStreamSynchronize(h->stream));
    return OD_OK;
}

int od_density_read(od_handle* h, uint64_t* counts, double* density, int64_t* samples)
{
    if (!h) return fail(h, OD_EINVAL, "bad handle");
    if (!h->d_hist) return fail(h, OD_EINVAL, "no density map: call od_density_enable first");
    const int nr = h->hist_nr, nz = h->hist_nz;
    std::vector<unsigned long long> c((size_t)nr * nz);
    OD_CK(h, cudaMemcpyAsync(c.data(), h->d_hist, sizeof(unsigned long long) * c.size(), cudaMemcpyDeviceToHost,
                             h->stream));
    OD_CK(h, cudaStreamSynchronize(h->stream));
    if (counts) std::memcpy(counts, c.data(), sizeof(uint64_t) * c.size());
    if (samples) *samples = h->hist_samples;
    if (density) {
        const double R = h->P.R, dz = h->P.H / nz, w = h->prm.weight > 0 ? h->prm.weight : 1.0;
        for (int iz = 0; iz < nz; ++iz)
            for (int ir = 0; ir < nr; ++ir) {
                const double r0 = R * ir / nr, r1 = R * (ir + 1) / nr;
                const double vol = 3.141592653589793 * (r1 * r1 - r0 * r0) * dz;
                density[(size_t)iz * nr + ir] =
                    h->hist_samples > 0 ? (double)c[(size_t)iz * nr + ir] * w / (h->hist_samples * vol) : 0.0;
            }
    }
    return OD_OK;
}

int od_write_ions(od_handle* h, const char* path, int32_t format)
{
    if (!h || !path || (format != OD_DUMP_XYZ && format != OD_DUMP_CSV)) return fail(h, OD_EINVAL, "bad argument");
    const long long N = h->P.N;
    std::vector<double> x(3 * (size_t)std::max(N, 1ll)), v(x.size());
    std::vector<uint64_t> id((size_t)std::max(N, 1ll));
    const int64_t got = od_get_ions(h, x.data(), v.data(), nullptr, id.data(), N);
    if (got < 0) return (int)got;
    FILE* f = std::fopen(path, "w");
    if (!f) return fail(h, OD_EINVAL, std::string("cannot open ") + path);
    if (format == OD_DUMP_XYZ) {
        std::fprintf(f, "%lld\n", N);
        std::fprintf(f, "Properties=species:S:1:pos:R:3:vel:R:3:id:I:1 step=%lld time=%.17g units=SI\n", h->host_step,
                     h->host_step * h->P.dt);
        for (long long i = 0; i < N; ++i)
            std::fprintf(f, "I %.17g %.17g %.17g %.17g %.17g %.17g %llu\n", x[3 * i], x[3 * i + 1], x[3 * i + 2],
                         v[3 * i], v[3 * i + 1], v[3 * i + 2], (unsigned long long)id[i]);
    } else {
        std::fprintf(f, "id,x,y,z,vx,vy,vz\n");
        for (long long i = 0; i < N; ++i)
            std::fprintf(f, "%llu,%.17g,%.17g,%.17g,%.17g,%.17g,%.17g\n", (unsigned long long)id[i], x[3 * i],
                         x[3 * i + 1], x[3 * i + 2], v[3 * i], v[3 * i + 1], v[3 * i + 2]);
    }
    const bool ok = std::fclose(f) == 0;
    return ok ? OD_OK : fail(h, OD_EINVAL, std::string("write failed: ") + path);
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

static const int kTuneGrains[4] = {4, 8, 16, 32};
static const int kTuneBps[3] = {0, 4, 2};  // persistent CTAs per SM: 0 = occupancy limit

static int apply_force_config(od_handle* h, int variant, int upb, int bps)
{
    h->variant = variant;
    h->upb = upb;
    h->bps = bps;
    int rc = replan(h, h->P.N);
    if (rc) return rc;
    h->graph_ok = false;
    // the padded length may have grown: rewrite positions and far-away dummies
    OD_LK(h, launch_fpos(h->P, h->B, (int)(h->host_step & 1), h->stream));
    return OD_OK;
}

int od_set_force_config(od_handle* h, int variant, int units_per_block, int blocks_per_sm)
{
    if (!h || variant < 0 || variant >= num_force_variants() || units_per_block < 1 || units_per_block > 1024 ||
        blocks_per_sm < 0 || blocks_per_sm > 64 || h->batch_member)
        return fail(h, OD_EINVAL, "bad force configuration (or a batch member: use od_batch_set_config)");
    int rc = apply_force_config(h, variant, units_per_block, blocks_per_sm);
    if (rc) return rc;
    OD_CK(h, cudaStreamSynchronize(h->stream));
    return OD_OK;
}

int od_tune(od_handle* h, int reps, double* ms, int* best_variant, int* best_upb, int* best_bps)
{
    if (!h || reps < 1 || h->batch_member)
        return fail(h, OD_EINVAL, "bad handle or repetition count (or a batch member: use od_batch_tune)");
    if (h->cut_on) return fail(h, OD_EINVAL, "the cutoff has a fixed plan: switch it off to tune the all-pairs kernels");
    if (h->P.flags & OD_F_FP64_PAIRS) return fail(h, OD_EINVAL, "the FP64 study kernel has no variants to tune");
    const int nv = num_force_variants();
    if (ms)
        for (int i = 0; i < nv * 4 * 3; ++i) ms[i] = -1.0;
    if (h->P.N == 0 || (h->P.flags & OD_F_NO_IONION)) {
        if (best_variant) *best_variant = h->variant;
        if (best_upb) *best_upb = h->upb;
        if (best_bps) *best_bps = h->bps;
        return OD_OK;
    }
    double best = 1e300;
    int bv = h->variant, bg = h->upb, bb = h->bps;
    size_t free_b = 0, total_b = 0;
    OD_CK(h, cudaMemGetInfo(&free_b, &total_b));
    const double slot_budget = (double)(free_b + sizeof(float4) * (size_t)h->part_cap) / 8.0;
    for (int v = 0; v < nv; ++v)
        for (int g = 0; g < 4; ++g)
            for (int c = 0; c < 3; ++c) {
                if (kTuneBps[c] >= force_blocks_per_sm(v)) continue;  // no cap below the occupancy limit
                const ForceVariant fv = force_variant(v);
                if (fv.sym) {
                    if (g > 0) continue;  // fixed-size units: one grain setting
                    // one partial slot per tile for every ion: skip layouts that would take
                    // more than an eighth of the device memory
                    const double ti = fv.BT * fv.IPT, np = std::ceil(h->P.N / ti) * ti;
                    if (np / ti * np * sizeof(float4) > slot_budget) continue;
                }
                int rc = apply_force_config(h, v, kTuneGrains[g], kTuneBps[c]);
                if (rc) return rc;
                // the kick is timed too: it sums every ion's partial slots, one per tile
                // for the symmetric kernel
                OD_LK(h, launch_forces(h->P, h->B, h->F, h->variant, h->stream));
                OD_CK(h, cudaEventRecord(h->ev[0], h->stream));
                for (int r = 0; r < reps; ++r) {
                    OD_LK(h, launch_forces(h->P, h->B, h->F, h->variant, h->stream));
                    OD_LK(h, launch_kick(h->P, h->B, h->F, 1, h->stream));
                }
                OD_CK(h, cudaEventRecord(h->ev[1], h->stream));
                OD_CK(h, cudaEventSynchronize(h->ev[1]));
                float t = 0.f;
                OD_CK(h, cudaEventElapsedTime(&t, h->ev[0], h->ev[1]));
                const double avg = t / reps;
                if (ms) ms[(v * 4 + g) * 3 + c] = avg;
                if (avg < best) {
                    best = avg;
                    bv = v;
                    bg = kTuneGrains[g];
                    bb = kTuneBps[c];
                }
            }
    int rc = apply_force_config(h, bv, bg, bb);
    if (rc) return rc;
    // give back partial-slot memory beyond what the chosen layout needs
    if (h->part_cap > 2 * (long long)h->F.W * h->F.n_pad) {
        OD_CK(h, cudaStreamSynchronize(h->stream));
        cudaFree(h->B.part);
        h->B.part = nullptr;
        h->part_cap = 0;
        if ((rc = ensure_part(h))) return rc;
    }
    // the accelerations and partial sums left by the timing belong to other kernels:
    // evaluate the current state again with the chosen one
    if ((rc = force_eval(h))) return rc;
    OD_CK(h, cudaStreamSynchronize(h->stream));
    if (best_variant) *best_variant = bv;
    if (best_upb) *best_upb = bg;
    if (best_bps) *best_bps = bb;
    return read_error_word(h);
}

int od_selftest_wait_timeout(od_handle* h, int64_t polls)
{
    if (!h || polls < 1) return fail(h, OD_EINVAL, "bad handle or poll limit");
    if (h->P.N <= push_tile()) return fail(h, OD_EINVAL, "the wait self-test needs more than one scan tile");
    Phys P = h->P;
    P.spin_limit = polls;
    P.test_hold_tile0 = 1;
    OD_LK(h, launch_push_scan(P, h->B, h->stream));
    OD_CK(h, cudaStreamSynchronize(h->stream));
    h->graph_ok = false;
    return read_error_word(h);
}

int od_get_force_config(od_handle* h, int* variant, int* units_per_block, int* blocks_per_sm, int* n_variants)
{
    if (!h) return fail(h, OD_EINVAL, "bad handle");
    if (variant) *variant = h->variant;
    if (units_per_block) *units_per_block = h->upb;
    if (blocks_per_sm) *blocks_per_sm = h->bps;
    if (n_variants) *n_variants = num_force_variants();
    return OD_OK;
}

int od_num_dust(od_handle* h) { return h ? h->P.D : fail(h, OD_EINVAL, "bad handle"); }

// ------------------------------------------------------------------ checkpoints
// File layout (host byte order): CkptHeader, then x[N][3], v[N][3] (double), id[N]
// (uint64), acc[N] (float x4), the control block (ctrl_bytes), the per-step records
// double[n_series][OD_MAX_DUST][OD_REC] and events int32[n_series][OD_EV].
struct CkptHeader {
    char magic[8];
    uint32_t version, header_bytes;
    double ion_mass, ion_charge_number, T_i, T_n, T_e, n_inf, mach, E_ext, nu_in, R, H, dt, weight;
    int64_t n_ions;
    int32_t n_dust, charge_model;
    uint64_t seed;
    int64_t avg_start;
    int32_t flags, eout_grid;
    od_dust dust[OD_MAX_DUST];
    double alpha[15];
    int64_t N, step;
    int32_t variant, upb, bps, pad;
    int64_t n_series;
    uint64_t ctrl_bytes;
    double r_cut, r_switch;  // ion-ion cutoff (0: none)
};
static const char kCkptMagic[8] = {'O', 'D', 'C', 'K', 'P', 'T', '0', '1'};

int od_save(od_handle* h, const char* path)
{
    if (!h || !path) return fail(h, OD_EINVAL, "bad argument");
    if (h->batch_member) return fail(h, OD_EINVAL, "batch members are saved through their own runs' state only");
    const long long N = h->P.N;
    CkptHeader hd{};
    std::memcpy(hd.magic, kCkptMagic, 8);
    hd.version = 1;
    hd.header_bytes = sizeof(CkptHeader);
    const od_params& p = h->prm;
    hd.ion_mass = p.ion_mass, hd.ion_charge_number = p.ion_charge_number, hd.T_i = p.T_i, hd.T_n = p.T_n;
    hd.T_e = p.T_e, hd.n_inf = p.n_inf, hd.mach = p.mach, hd.E_ext = p.E_ext, hd.nu_in = p.nu_in;
    hd.R = p.R, hd.H = p.H, hd.dt = p.dt, hd.weight = p.weight, hd.n_ions = p.n_ions;
    hd.n_dust = p.n_dust, hd.charge_model = p.charge_model, hd.seed = p.seed, hd.avg_start = p.avg_start;
    hd.flags = p.flags, hd.eout_grid = p.eout_grid;
    for (int k = 0; k < p.n_dust; ++k) hd.dust[k] = h->prm_dust[k];
    for (int t = 0; t < 15; ++t) hd.alpha[t] = h->alpha[t];
    hd.N = N;
    hd.step = h->host_step;
    hd.variant = h->variant, hd.upb = h->upb, hd.bps = h->bps;
    hd.n_series = std::min<long long>(h->host_step, h->series_cap);
    hd.ctrl_bytes = sizeof(Ctrl);
    hd.r_cut = h->cut_on ? h->r_cut : 0.0;
    hd.r_switch = h->cut_on ? h->r_switch : 0.0;
    std::vector<double> x(3 * (size_t)std::max(N, 1ll)), v(x.size());
    std::vector<uint64_t> id((size_t)std::max(N, 1ll));
    const int64_t got = od_get_ions(h, x.data(), v.data(), nullptr, id.data(), N);
    if (got < 0) return (int)got;
    std::vector<float4> acc((size_t)std::max(N, 1ll));
    Ctrl c;
    std::vector<double> ser((size_t)hd.n_series * MAXD * REC);
    std::vector<int> evs((size_t)hd.n_series * EV);
    if (N > 0) OD_CK(h, cudaMemcpyAsync(acc.data(), h->B.acc, sizeof(float4) * N, cudaMemcpyDeviceToHost, h->stream));
    OD_CK(h, cudaMemcpyAsync(&c, h->B.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
    if (hd.n_series > 0) {
        OD_CK(h, cudaMemcpyAsync(ser.data(), h->d_series, sizeof(double) * ser.size(), cudaMemcpyDeviceToHost, h->stream));
        OD_CK(h, cudaMemcpyAsync(evs.data(), h->d_evseries, sizeof(int) * evs.size(), cudaMemcpyDeviceToHost, h->stream));
    }
    OD_CK(h, cudaStreamSynchronize(h->stream));
    c.series = nullptr;  // device addresses mean nothing in a file
    c.evseries = nullptr;
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(h, OD_EINVAL, std::string("cannot open ") + path);
    bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1;
    ok = ok && (N == 0 || (std::fwrite(x.data(), sizeof(double), 3 * N, f) == (size_t)(3 * N) &&
                           std::fwrite(v.data(), sizeof(double), 3 * N, f) == (size_t)(3 * N) &&
                           std::fwrite(id.data(), sizeof(uint64_t), N, f) == (size_t)N &&
                           std::fwrite(acc.data(), sizeof(float4), N, f) == (size_t)N));
    ok = ok && std::fwrite(&c, sizeof(Ctrl), 1, f) == 1;
    ok = ok && (ser.empty() || std::fwrite(ser.data(), sizeof(double), ser.size(), f) == ser.size());
    ok = ok && (evs.empty() || std::fwrite(evs.data(), sizeof(int), evs.size(), f) == evs.size());
    ok = (std::fclose(f) == 0) && ok;
    return ok ? OD_OK : fail(h, OD_EINVAL, std::string("write failed: ") + path);
}

int od_load(const char* path, void* cuda_stream, od_handle** out)
{
    if (!out || !path) return fail(nullptr, OD_EINVAL, "bad argument");
    *out = nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(nullptr, OD_EINVAL, std::string("cannot open ") + path);
    CkptHeader hd{};
    auto bad = [&](const std::string& m) {
        std::fclose(f);
        return fail(nullptr, OD_EINVAL, "not a checkpoint of this library (" + m + "): " + path);
    };
    if (std::fread(&hd, sizeof(hd), 1, f) != 1) return bad("short header");
    if (std::memcmp(hd.magic, kCkptMagic, 8) != 0) return bad("magic");
    if (hd.version != 1 || hd.header_bytes != sizeof(CkptHeader) || hd.ctrl_bytes != sizeof(Ctrl))
        return bad("version or layout");
    if (hd.N < 0 || hd.step < 0 || hd.n_series < 0 || hd.n_series > hd.step || hd.n_dust < 0 || hd.n_dust > OD_MAX_DUST)
        return bad("sizes");
    const long long N = hd.N;
    std::vector<double> x(3 * (size_t)std::max(N, 1ll)), v(x.size());
    std::vector<uint64_t> id((size_t)std::max(N, 1ll));
    std::vector<float4> acc((size_t)std::max(N, 1ll));
    Ctrl c;
    std::vector<double> ser((size_t)hd.n_series * MAXD * REC);
    std::vector<int> evs((size_t)hd.n_series * EV);
    bool ok = N == 0 || (std::fread(x.data(), sizeof(double), 3 * N, f) == (size_t)(3 * N) &&
                         std::fread(v.data(), sizeof(double), 3 * N, f) == (size_t)(3 * N) &&
                         std::fread(id.data(), sizeof(uint64_t), N, f) == (size_t)N &&
                         std::fread(acc.data(), sizeof(float4), N, f) == (size_t)N);
    ok = ok && std::fread(&c, sizeof(Ctrl), 1, f) == 1;
    ok = ok && (ser.empty() || std::fread(ser.data(), sizeof(double), ser.size(), f) == ser.size());
    ok = ok && (evs.empty() || std::fread(evs.data(), sizeof(int), evs.size(), f) == evs.size());
    if (!ok) return bad("truncated");
    std::fclose(f);
    if (c.step != hd.step) return fail(nullptr, OD_EINVAL, std::string("inconsistent checkpoint: ") + path);
    od_params p{};
    p.ion_mass = hd.ion_mass, p.ion_charge_number = hd.ion_charge_number, p.T_i = hd.T_i, p.T_n = hd.T_n;
    p.T_e = hd.T_e, p.n_inf = hd.n_inf, p.mach = hd.mach, p.E_ext = hd.E_ext, p.nu_in = hd.nu_in;
    p.R = hd.R, p.H = hd.H, p.dt = hd.dt, p.weight = hd.weight;
    p.n_ions = N > 0 ? N : hd.n_ions;
    p.n_dust = hd.n_dust, p.charge_model = hd.charge_model, p.dust = hd.dust, p.seed = hd.seed;
    p.avg_start = hd.avg_start, p.eout_coeffs = hd.alpha, p.flags = hd.flags, p.eout_grid = hd.eout_grid;
    p.cuda_stream = cuda_stream;
    od_handle* h = nullptr;
    int rc = od_create(&p, &h);
    if (rc) return rc;
    auto done = [&](int code) {
        if (code) {
            g_create_error = h->err;
            od_destroy(h);
        } else {
            *out = h;
        }
        return code;
    };
    // the creation parameters as saved (n_ions as given originally)
    h->prm.n_ions = hd.n_ions;
    if (hd.r_cut > 0.0 && (rc = od_set_cutoff(h, hd.r_cut, hd.r_switch))) return done(rc);
    h->host_step = hd.step;
    const int buf = (int)(hd.step & 1);
    if (N > 0) {
        std::vector<double> tmp(3 * (size_t)N);
        for (int which = 0; which < 2; ++which) {
            const double* src = which == 0 ? x.data() : v.data();
            double* d = which == 0 ? h->B.x[buf] : h->B.v[buf];
            for (long long i = 0; i < N; ++i)
                for (int k = 0; k < 3; ++k) tmp[k * N + i] = src[3 * i + k];
            for (int k = 0; k < 3; ++k)
                if (cudaMemcpyAsync(d + k * h->cap, tmp.data() + k * N, sizeof(double) * N, cudaMemcpyHostToDevice,
                                    h->stream) != cudaSuccess)
                    return done(fail(h, OD_ECUDA, "checkpoint upload failed"));
            if (cudaStreamSynchronize(h->stream) != cudaSuccess) return done(fail(h, OD_ECUDA, "checkpoint upload failed"));
        }
        if (cudaMemcpyAsync(h->B.id[buf], id.data(), sizeof(uint64_t) * N, cudaMemcpyHostToDevice, h->stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(h->B.acc, acc.data(), sizeof(float4) * N, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
            return done(fail(h, OD_ECUDA, "checkpoint upload failed"));
    }
    if ((rc = ensure_series(h, std::max<long long>(hd.n_series, 1)))) return done(rc);
    if (hd.n_series > 0 &&
        (cudaMemcpyAsync(h->d_series, ser.data(), sizeof(double) * ser.size(), cudaMemcpyHostToDevice, h->stream) !=
             cudaSuccess ||
         cudaMemcpyAsync(h->d_evseries, evs.data(), sizeof(int) * evs.size(), cudaMemcpyHostToDevice, h->stream) !=
             cudaSuccess))
        return done(fail(h, OD_ECUDA, "checkpoint upload failed"));
    c.series = h->d_series;
    c.evseries = h->d_evseries;
    c.series_cap = h->series_cap;
    if (cudaMemcpyAsync(h->B.ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
        return done(fail(h, OD_ECUDA, "checkpoint upload failed"));
    // the pair kernel that produced the saved state, so that the continuation is exact
    if (hd.variant >= 0 && hd.variant < num_force_variants()) {
        if ((rc = apply_force_config(h, hd.variant, hd.upb, hd.bps))) return done(rc);
    } else {
        if ((rc = replan(h, plan_n(h, N)))) return done(rc);
        if (launch_fpos(h->P, h->B, buf, h->stream)) return done(fail(h, OD_ECUDA, "position refresh failed"));
    }
    h->graph_ok = false;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return done(fail(h, OD_ECUDA, "checkpoint upload failed"));
    return done(read_error_word(h));
}

}  // extern "C"

// ------------------------------------------------------------------ batches
struct od_batch {
    std::vector<od_handle*> runs;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    RunDesc* d_runs = nullptr;
    int2* d_tasks = nullptr;
    int2* d_tasks_f = nullptr;          // tuning: pair units, then kick tiles
    unsigned long long* d_done = nullptr;
    unsigned long long* d_done_f = nullptr;  // phase counters of the tuning launches
    BatchCtrl* d_bc = nullptr;
    BatchCtrl* d_bc_f = nullptr;
    long long T = 0, T_f = 0;
    int4 phase_end{0, 0, 0, 0}, phase_end_f{0, 0, 0, 0};
    int ipt = 2, jc = 4096, grid = 1, sms = 1;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool graph_ok = false;
    long long host_step = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::string err;
};

namespace {

thread_local std::string g_batch_error;

int bfail(od_batch* b, int code, const std::string& msg)
{
    if (b) b->err = msg;
    else g_batch_error = msg;
    return code;
}

#define OD_BCK(b, call)                                                                              \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? OD_ENOMEM : OD_ECUDA,                  \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                        \
    } while (0)

// apply the batch pair plan (ipt, jc) to every run and rebuild the task lists
int batch_build(od_batch* b)
{
    const int R = (int)b->runs.size();
    std::vector<RunDesc> desc(R);
    std::vector<int2> tA, tF, tK, tD;
    for (int r = 0; r < R; ++r) {
        od_handle* h = b->runs[r];
        h->F = batch_plan(h->P.N, b->ipt, b->jc);
        h->P.n_pad = h->F.n_pad;
        if (h->F.n_pad > h->npad_cap) return bfail(b, OD_EOVERFLOW, "padded ion count exceeds a run's buffer");
        int rc = ensure_part(h);
        if (rc) return bfail(b, rc, h->err);
        rc = launch_fpos(h->P, h->B, (int)(h->host_step & 1), b->stream);
        if (rc) return bfail(b, OD_ECUDA, "batch: position refresh failed");
        desc[r].P = h->P;
        desc[r].B = h->B;
        desc[r].F = h->F;
        desc[r].nA = (h->P.N + BATCH_TILE - 1) / BATCH_TILE;
        desc[r].nK = desc[r].nA;
        for (int i = 0; i < desc[r].nA; ++i) tA.push_back(make_int2(r, i));
        for (long long u = 0; u < h->F.U; ++u) tF.push_back(make_int2(r, (int)u));
        for (int i = 0; i < desc[r].nK; ++i) tK.push_back(make_int2(r, i));
        tD.push_back(make_int2(r, 0));
    }
    std::vector<int2> all;
    all.insert(all.end(), tA.begin(), tA.end());
    all.insert(all.end(), tF.begin(), tF.end());
    all.insert(all.end(), tK.begin(), tK.end());
    all.insert(all.end(), tD.begin(), tD.end());
    b->phase_end = make_int4((int)tA.size(), (int)(tA.size() + tF.size()), (int)(tA.size() + tF.size() + tK.size()),
                             (int)all.size());
    b->T = (long long)all.size();
    std::vector<int2> fk(tF);
    fk.insert(fk.end(), tK.begin(), tK.end());
    b->phase_end_f = make_int4(0, (int)tF.size(), (int)fk.size(), (int)fk.size());
    b->T_f = (long long)fk.size();
    cudaFree(b->d_runs);
    cudaFree(b->d_tasks);
    cudaFree(b->d_tasks_f);
    b->d_runs = nullptr;
    b->d_tasks = b->d_tasks_f = nullptr;
    OD_BCK(b, cudaMalloc(&b->d_runs, sizeof(RunDesc) * R));
    OD_BCK(b, cudaMalloc(&b->d_tasks, sizeof(int2) * std::max<size_t>(all.size(), 1)));
    OD_BCK(b, cudaMalloc(&b->d_tasks_f, sizeof(int2) * std::max<size_t>(fk.size(), 1)));
    OD_BCK(b, cudaMemcpyAsync(b->d_runs, desc.data(), sizeof(RunDesc) * R, cudaMemcpyHostToDevice, b->stream));
    OD_BCK(b, cudaMemcpyAsync(b->d_tasks, all.data(), sizeof(int2) * all.size(), cudaMemcpyHostToDevice, b->stream));
    if (!fk.empty())
        OD_BCK(b, cudaMemcpyAsync(b->d_tasks_f, fk.data(), sizeof(int2) * fk.size(), cudaMemcpyHostToDevice, b->stream));
    b->grid = (int)std::max(1ll, std::min<long long>((long long)batch_blocks_per_sm(b->ipt) * b->sms, b->T));
    OD_BCK(b, cudaStreamSynchronize(b->stream));
    b->graph_ok = false;
    return OD_OK;
}

void batch_free(od_batch* b)
{
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (od_handle* h : b->runs) {
        free_all(h);
        delete h;
    }
    cudaFree(b->d_runs);
    cudaFree(b->d_tasks);
    cudaFree(b->d_tasks_f);
    cudaFree(b->d_done);
    cudaFree(b->d_done_f);
    cudaFree(b->d_bc);
    cudaFree(b->d_bc_f);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->e0) cudaEventDestroy(b->e0);
    if (b->e1) cudaEventDestroy(b->e1);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

int batch_check(od_batch* b)
{
    BatchCtrl bc;
    OD_BCK(b, cudaMemcpyAsync(&bc, b->d_bc, sizeof(bc), cudaMemcpyDeviceToHost, b->stream));
    OD_BCK(b, cudaStreamSynchronize(b->stream));
    if (bc.err & ERR_TIMEOUT) return bfail(b, OD_ETIMEOUT, "batch: a task's dependency wait hit its limit");
    for (size_t r = 0; r < b->runs.size(); ++r) {
        const int rc = read_error_word(b->runs[r]);
        if (rc) return bfail(b, rc, "run " + std::to_string(r) + ": " + b->runs[r]->err);
    }
    return OD_OK;
}

}  // namespace

extern "C" {

int od_create_batch(const od_params* ps, int32_t R, od_batch** out)
{
    if (!out || !ps || R < 1) return bfail(nullptr, OD_EINVAL, "bad batch arguments");
    *out = nullptr;
    for (int r = 0; r < R; ++r) {
        std::string msg;
        const int rc = validate(ps + r, msg);
        if (rc) return bfail(nullptr, rc, "run " + std::to_string(r) + ": " + msg);
        if (ps[r].flags & OD_F_FLUX_INJECT)
            return bfail(nullptr, OD_EINVAL, "run " + std::to_string(r) + ": batched runs keep a fixed ion count");
        if (ps[r].flags & OD_F_FP64_PAIRS)
            return bfail(nullptr, OD_EINVAL, "run " + std::to_string(r) + ": the FP64 study kernel runs alone");
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return bfail(nullptr, OD_ENODEV, "no CUDA device");
    od_batch* b = new od_batch();
    int rc = OD_OK;
    auto fail_out = [&](int code) {
        g_batch_error = b->err;
        batch_free(b);
        delete b;
        return code;
    };
    if (ps[0].cuda_stream) {
        b->stream = (cudaStream_t)ps[0].cuda_stream;
    } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        b->err = "stream creation failed";
        return fail_out(OD_ECUDA);
    } else {
        b->own_stream = true;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    for (int r = 0; r < R; ++r) {
        od_params p = ps[r];
        p.cuda_stream = b->stream;
        od_handle* h = new od_handle();
        h->batch_member = true;
        rc = create_impl(&p, h);
        if (rc) {
            b->err = "run " + std::to_string(r) + ": " + h->err;
            free_all(h);
            delete h;
            return fail_out(rc);
        }
        h->batch_member = true;
        h->own_stream = false;
        b->runs.push_back(h);
    }
    if (cudaMalloc(&b->d_done, sizeof(unsigned long long) * 3 * R) != cudaSuccess ||
        cudaMalloc(&b->d_done_f, sizeof(unsigned long long) * 3 * R) != cudaSuccess ||
        cudaMalloc(&b->d_bc, sizeof(BatchCtrl)) != cudaSuccess || cudaMalloc(&b->d_bc_f, sizeof(BatchCtrl)) != cudaSuccess ||
        cudaEventCreate(&b->e0) != cudaSuccess || cudaEventCreate(&b->e1) != cudaSuccess) {
        b->err = "batch allocation failed";
        return fail_out(OD_ENOMEM);
    }
    cudaMemsetAsync(b->d_done, 0, sizeof(unsigned long long) * 3 * R, b->stream);
    cudaMemsetAsync(b->d_bc, 0, sizeof(BatchCtrl), b->stream);
    rc = batch_build(b);
    if (rc) return fail_out(rc);
    *out = b;
    return OD_OK;
}

int od_batch_step(od_batch* b, int64_t n)
{
    if (!b || n < 0) return bfail(b, OD_EINVAL, "bad batch or step count");
    if (n == 0) return OD_OK;
    for (od_handle* h : b->runs) {
        const int rc = ensure_series(h, h->host_step + n);
        if (rc) return bfail(b, rc, h->err);
    }
    if (!b->graph_ok) {
        if (b->gexec) cudaGraphExecDestroy(b->gexec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->gexec = nullptr;
        b->graph = nullptr;
        OD_BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        const int lrc = launch_batch(b->ipt, b->grid, b->d_runs, b->d_tasks, b->phase_end, b->T, b->d_bc, b->d_done,
                                     (int)b->runs.size(), SPIN_LIMIT, 0, b->stream);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (lrc) return bfail(b, OD_ECUDA, std::string("batch launch: ") + cudaGetErrorString((cudaError_t)lrc));
        if (e != cudaSuccess) return bfail(b, OD_ECUDA, std::string("batch capture: ") + cudaGetErrorString(e));
        b->graph = g;
        OD_BCK(b, cudaGraphInstantiate(&b->gexec, g, 0));
        b->graph_ok = true;
    }
    for (int64_t s = 0; s < n; ++s) OD_BCK(b, cudaGraphLaunch(b->gexec, b->stream));
    for (od_handle* h : b->runs) h->host_step += n;
    b->host_step += n;
    return batch_check(b);
}

od_handle* od_batch_run(od_batch* b, int32_t r)
{
    if (!b || r < 0 || r >= (int)b->runs.size()) return nullptr;
    return b->runs[r];
}

int od_batch_size(const od_batch* b) { return b ? (int)b->runs.size() : 0; }

// one tuning launch of the current plan: every run's pair units, then its kick tiles in
// forces-only mode (fresh counters per configuration)
static int batch_tune_launch(od_batch* b, int grid)
{
    const int lrc = launch_batch(b->ipt, grid, b->d_runs, b->d_tasks_f, b->phase_end_f, b->T_f, b->d_bc_f,
                                 b->d_done_f, (int)b->runs.size(), SPIN_LIMIT, 1, b->stream);
    return lrc ? bfail(b, OD_ECUDA, "batch tune launch failed") : OD_OK;
}

int od_batch_tune(od_batch* b, int reps, double* ms, int* best_ipt, int* best_jc)
{
    if (!b || reps < 1) return bfail(b, OD_EINVAL, "bad batch or repetition count");
    static const int ipts[3] = {1, 2, 4};
    static const int jcs[4] = {2048, 4096, 8192, 0};  // 0: symmetric tile pairs
    double best = 1e300;
    int bi = b->ipt, bj = b->jc;
    const int R = (int)b->runs.size();
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 4; ++c) {
            b->ipt = ipts[a];
            b->jc = jcs[c];
            int rc = batch_build(b);
            if (rc) return rc;
            OD_BCK(b, cudaMemsetAsync(b->d_bc_f, 0, sizeof(BatchCtrl), b->stream));
            OD_BCK(b, cudaMemsetAsync(b->d_done_f, 0, sizeof(unsigned long long) * 3 * R, b->stream));
            const int grid = (int)std::max(1ll, std::min<long long>((long long)batch_blocks_per_sm(b->ipt) * b->sms, b->T_f));
            if ((rc = batch_tune_launch(b, grid))) return rc;
            OD_BCK(b, cudaEventRecord(b->e0, b->stream));
            for (int i = 0; i < reps; ++i)
                if ((rc = batch_tune_launch(b, grid))) return rc;
            OD_BCK(b, cudaEventRecord(b->e1, b->stream));
            OD_BCK(b, cudaEventSynchronize(b->e1));
            float t = 0.f;
            OD_BCK(b, cudaEventElapsedTime(&t, b->e0, b->e1));
            if (ms) ms[a * 4 + c] = t / reps;
            if (t / reps < best) {
                best = t / reps;
                bi = ipts[a];
                bj = jcs[c];
            }
        }
    b->ipt = bi;
    b->jc = bj;
    int rc = batch_build(b);
    if (rc) return rc;
    // the accelerations left by the timing belong to other plans: evaluate them again
    // with the chosen one
    OD_BCK(b, cudaMemsetAsync(b->d_bc_f, 0, sizeof(BatchCtrl), b->stream));
    OD_BCK(b, cudaMemsetAsync(b->d_done_f, 0, sizeof(unsigned long long) * 3 * R, b->stream));
    if ((rc = batch_tune_launch(b, (int)std::max(1ll, std::min<long long>((long long)batch_blocks_per_sm(b->ipt) * b->sms,
                                                                            b->T_f)))))
        return rc;
    if ((rc = batch_check(b))) return rc;
    if (best_ipt) *best_ipt = bi;
    if (best_jc) *best_jc = bj;
    return OD_OK;
}

int od_batch_set_config(od_batch* b, int ipt, int jc)
{
    if (!b || (ipt != 1 && ipt != 2 && ipt != 4) || (jc != 0 && jc < 256))
        return bfail(b, OD_EINVAL, "bad batch configuration");
    b->ipt = ipt;
    b->jc = jc;
    return batch_build(b);
}

void od_destroy_batch(od_batch* b)
{
    if (!b) return;
    batch_free(b);
    delete b;
}

const char* od_batch_last_error(const od_batch* b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

}  // extern "C"
