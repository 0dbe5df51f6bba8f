// Host-side internals shared by the translation units of the C ABI: the run handle and
// the helpers that derive, plan, launch and check its work (od_api.cu), configure its
// pair kernels (od_config.cu), save and load it (od_io.cu) and step it in batches
// (od_batch_api.cu).
#pragma once

#include <string>
#include <vector>

#include "od_internal.h"

constexpr int PROF_RING = 64;  // steps per read of the profiling events
constexpr int STEP_GRAPH_K = 16;  // steps in the long step graph

struct od_handle {
    od::Phys P{};
    od::Bufs B{};
    od::ForceArgs F{};
    float qscale = 1.f;  // 2^K of the fixed-point pair sums
    int variant = 0;
    int upb = 8;  // pair-kernel work units per persistent block
    int bps = 0;  // persistent pair-kernel CTAs per SM (0 = occupancy limit)
    bool batch_member = false;  // stepped only through its batch (od_batch_step)
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t aux = nullptr;   // next step's injection samples beside the pair forces
    cudaStream_t aux2 = nullptr;  // this step's collision velocities beside the pair forces
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool graph_ok = false;  // false: both step graphs are recaptured before the next step
    cudaGraph_t graph_k = nullptr;  // STEP_GRAPH_K steps in one graph (long od_step calls)
    cudaGraphExec_t gexec_k = nullptr;
    bool graph_k_ok = false;
    long long cap = 0;       // ion capacity
    long long npad_cap = 0;  // fpos capacity
    long long part_cap = 0;  // partial-sum capacity (float4)
    long long nb_cap = 0;    // kick blocks capacity
    long long scan_tiles_cap = 0;  // scan tile status words (tiles of the smaller of the single-run and batch scan)
    long long host_step = 0;
    long long series_cap = 0;
    int sms = 0;
    double alpha[15] = {0};
    double info[32] = {0};
    std::string err;
    bool profiling = false;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    std::vector<cudaEvent_t> pev;  // profiling: 5 events per step for up to PROF_RING steps
    int pev_used = 0;              // steps recorded in pev and not yet read
    double kms[4] = {0, 0, 0, 0};
    long long klaunch[4] = {0, 0, 0, 0};
    double* d_stats = nullptr;
    unsigned long long* d_sched = nullptr;  // unit queue of the symmetric and cutoff pair kernels
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
    od::CutBufs C{};
    int cut_grid = 1;
};

namespace od {
namespace host {

// CODATA 2018
constexpr double kQE = 1.602176634e-19;
constexpr double kKB = 1.380649e-23;
constexpr double kEPS0 = 8.8541878128e-12;
constexpr double kME = 9.1093837015e-31;
constexpr double kPI = 3.141592653589793238;
constexpr double kTWO32 = 4294967296.0;

extern thread_local std::string g_create_error;  // od_last_error(NULL)

int fail(od_handle* h, int code, const std::string& msg);
int cuda_fail(od_handle* h, cudaError_t e, const char* where);
int validate(const od_params* p, std::string& msg);
double oml_charge(const od_params* p, double a);
ForceArgs plan_forces(int N, int v, int sms, int units_per_block, int bps_cap);
int default_variant(int N);
int ensure_part(od_handle* h);
void attach_sums(const od_handle* h, ForceArgs& F);
int replan(od_handle* h, int N);
int launch_pairs(od_handle* h, int after_push);
int plan_n(const od_handle* h, long long n_live);
int read_error_word(od_handle* h);
int force_eval(od_handle* h);
int ensure_series(od_handle* h, long long need);
int ensure_io(od_handle* h);
bool host_pinned(const void* p);
void free_cut(od_handle* h);
void free_all(od_handle* h);
int create_impl(const od_params* p, od_handle* h);
int apply_force_config(od_handle* h, int variant, int upb, int bps);  // od_config.cu
void set_close_pairs(od_handle* h);                                   // od_config.cu

}  // namespace host
}  // namespace od

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
