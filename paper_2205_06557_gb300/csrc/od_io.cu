// Observability and restart of a run: checkpoints (od_save / od_load), ion dumps
// (od_write_ions) and the time-averaged density map (od_density_enable / _read).
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

extern "C" {

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
static const char kCkptMagic[8] = {'O', 'D', 'C', 'K', 'P', 'T', '0', '2'};

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
    c.ahead_n = 0;  // no injection samples computed ahead in this handle yet
    c.ahead_sn = 0;
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
