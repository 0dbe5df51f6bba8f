// Internal types of the GB300 ion-flow-around-dust library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "opendust.h"

namespace od {

constexpr int MAXD = OD_MAX_DUST;
constexpr int REC = OD_REC;
constexpr int EV = OD_EV;

// error bits of the device error word
constexpr int ERR_NAN = 1;
constexpr int ERR_TIMEOUT = 2;
constexpr int ERR_OVERFLOW = 4;
constexpr int ERR_PLACE = 8;
constexpr int ERR_RANGE = 32;   // a pair partial sum beyond the fixed-point range (ions nearly coincide)
constexpr long long SPIN_LIMIT = 1ll << 22;  // ~4 s of polling with the 1 us back-off
constexpr int VTAB_K = 4096;                  // intervals of the tabulated inverse flux CDFs
constexpr int INJ_AHEAD = 2048;               // injection samples computed one step ahead (at most)

// Philox streams (fourth counter word): the same layout on host and device.
enum : uint32_t {
    ST_INIT_POS = 0,
    ST_INIT_VEL = 1,
    ST_COLL = 2,
    ST_COLL_VEL = 3,
    ST_INJ_A = 4,
    ST_INJ_B = 5,
    ST_INJ_N = 6  // number of injections per step (flux rule)
};

// Device-resident control block: everything a step changes lives here, so a
// captured graph of one step can be replayed without host involvement.
struct Ctrl {
    long long step;               // steps completed
    unsigned long long next_id;   // id of the next injected ion
    int err;                      // ERR_* bits
    unsigned tile_counter;        // dynamic tile ids of the scan kernel
    unsigned done_counter;        // finished tiles of the scan kernel
    unsigned kick_done;           // finished blocks of the kick (the last one runs the grain tail)
    unsigned inj_done;            // finished blocks of the injection sampler (the last one tags)
    int removed_total;            // ions removed in the current step
    int ev_step[EV];              // this step's event counts
    int n_cur;                    // ions alive (N; varies with the flux injection rule)
    double Q[MAXD];               // grain charges
    double f_orbit[MAXD][3];      // Eq. 1 force at the last force evaluation
    double eg[MAXD][3];           // E_out at each grain's centre (App. A; set at creation)
    double wsum[MAXD][REC];       // window sums of the records
    long long wcount;             // records in the window
    long long counters[OD_NCOUNT];
    unsigned cp_epoch;            // close-pair cell lists: epoch of the last complete build (never 0)
    int ahead_n;                  // injection samples computed ahead: ids ahead_base + r, r < ahead_n,
    unsigned long long ahead_base;  // for step ahead_sn (0: none), in Bufs::inj_ahead
    long long ahead_sn;
    long long ahead_req_sn;       // the step the next samples are for (set by the scan's last tile)
    int ahead_want;               // how many to draw (the scan's estimate of the next step's need)
    int ahead_pad;
    double* series;               // [cap][MAXD][REC]
    int* evseries;                // [cap][EV]
    long long series_cap;
};

// Injected-ion staging (rank order) and removed-ion records (rank order)
struct Inj {
    double x, y, z, vx, vy, vz;
    unsigned long long id;
    int face;
    int pad;
};
struct Rem {
    double vx, vy, vz;
    int cls;  // -1 outflow, k >= 0 absorbed by grain k
    int pad;
};

// Physical constants and run parameters, passed by value to every kernel.
struct Phys {
    int N, n_pad, D, flags;  // N: ions the buffers and plans are sized for (with the flux
                             // injection rule a capacity above the live count Ctrl::n_cur)
    double inj_lambda;       // mean injections per step under the flux rule (App. B fluxes)
    double dt, R, H, hz, R2;
    double qm;       // Z e / m_i
    double kdi;      // Z e / (4 pi eps0 m_i): ion acceleration from a grain of charge Q
    double korb;     // q / (4 pi eps0): Eq. 1 prefactor per unit grain charge
    double lam_inv;  // 1 / lambda_De
    double E;        // driving field
    double m, q;     // superion mass and charge
    double sig, sig_n, u;
    float Ls_inv;    // log2(e) / lambda_De: scaled coordinates for the pair kernel
    float k_ii;      // q^2 / (4 pi eps0 m Ls^2), Ls = lambda_De / log2(e)
    uint32_t key0, key1;
    unsigned long long Tb, Tbt, Tcoll;
    double gx[MAXD], gy[MAXD], gz[MAXD], ga[MAXD], ga2[MAXD];
    // E_out = (-x G, -y G, -z K), G and K polynomials in r^2, z^2 (10 terms each)
    double Gc[10], Kc[10];
    int Gp[10], Gq[10], Kp[10], Kq[10];
    int eout;
    int charge_model;
    long long avg_start;
    double Ie0;      // OML electron flux at zero potential per unit area, 1/(m^2 s)
    double e_over_kTe;
    double inv4pieps0;
    // App. B inverse flux CDFs tabulated at U = k / VTAB_K (bottom face, then top face):
    // starting points and brackets for the Newton polish of every injected axial speed
    const double* vtab;
    double gmax_b, gmax_t;  // flux integrals G(v_max) and G_top(v_min) the CDFs are normalised by
    long long spin_limit;  // polls before a device-side wait gives up (ERR_TIMEOUT)
    int test_hold_tile0;   // wait self-test: the first scan tile never publishes its prefix
    // symmetric pair sums in fixed point: value x 2^K as int64 (qinv = 2^-K)
    double qinv;
    // close-pair correction of the FP32 position rounding: pairs closer than sqrt(cp_dc2)
    // (scaled units) found through hashed cells of side 1 / cp_hinv
    int cp_on;
    unsigned cp_mask;  // buckets - 1 (a power of two)
    float cp_hinv;
    double cp_dc2;
    double ls_inv;     // log2(e) / lambda_De in FP64
    int inj_ahead_flux;  // samples drawn ahead per step under the flux rule: lambda + 6 sqrt(lambda) + 32
    int inj_pad;
};

// Device buffers. Ion state is double-buffered (compaction writes the other copy).
struct Bufs {
    double* x[2];  // [3][cap] SoA: x, y, z
    double* v[2];  // [3][cap]
    unsigned long long* id[2];
    float4* acc;   // accelerations of the current order
    float4* fpos;  // scaled positions for the pair kernel, padded with far-away dummies
    float4* part;  // ordered pair-kernel partial sums [W][n_pad]
    long long* psum;  // symmetric pair sums in fixed point [3][psum_ld] (zero between evaluations)
    long long psum_ld;
    unsigned long long* cp_head;  // close-pair cell buckets: (epoch << 32) | first ion
    int* cp_next;                 // next ion of the same bucket, -1 at the end
    unsigned long long* tile_status;
    Inj* inj;
    Rem* rem;
    Inj* inj_ahead;  // [INJ_AHEAD] injection samples of the next step, computed during this one
    double* coll_v;  // [3][cap] neutral velocities of this step's colliding ions, computed beside the
                     // pair forces (null: the kick draws them)
    double* dpart; // grain partial sums [nb][MAXD][3]
    Ctrl* ctrl;
    long long cap;
};

// Balanced static partition of the all-pairs work into (i-tile, j-chunk) units.
struct ForceArgs {
    int n_pad;   // multiple of TI
    int TI;      // targets per tile = BT * IPT
    int JC;      // sources per chunk, multiple of BT
    int JS;      // chunks per tile
    int G;       // persistent blocks
    int W;       // partial slots (ordered kernel; 0 for the symmetric kernels)
    long long U; // units = n_itiles * JS (symmetric: T (T + 1) / 2 tile pairs)
    int sym;     // 1: symmetric kernel, JC = TI, JS = T tiles; sums go to the fixed-point
                 // accumulators psum (one int64 per ion and component, order-independent)
    long long* psum;
    long long psum_ld;
    float qscale;  // 2^K: a partial sum v adds round(v 2^K)
    int* err;      // the run's error word (ERR_RANGE)
    // ion-ion cutoff (symmetric tile pairs over z-sorted ions): switching zone in scaled
    // units [cut_s0, cut_s0 + 1 / cut_inv_w]; ion i sits at rank[i] in the sorted order,
    // which is also its accumulator index
    int cut;
    float cut_s0, cut_inv_w;
    const int* rank;
    // dynamic unit queue of the packed symmetric and cutoff kernels: [0] next unit,
    // [1] CTAs finished (both zero between launches)
    unsigned long long* sched;
    // live ion count (device; the plan covers the capacity under the flux rule), or null
    const int* n_live;
};

// One run of a batched launch (od_batch.cu): its parameters, buffers and pair plan.
struct RunDesc {
    Phys P;
    Bufs B;
    ForceArgs F;
    int nA;  // scan tiles (BATCH_TILE ions)
    int nK;  // kick tiles (BATCH_TILE ions)
};

// Device control block of a batched launch.
struct BatchCtrl {
    unsigned long long step;       // batched steps completed
    unsigned long long task_next;  // monotone task dispenser
    unsigned exit_count;
    int err;
};

constexpr int BATCH_TILE = 128;  // ions per scan / kick tile and threads per CTA of a batch
ForceArgs batch_plan(int N, int ipt, int jc);
int batch_blocks_per_sm(int ipt);
int launch_batch(int ipt, int grid, const RunDesc* runs, const int2* tasks, int4 phase_end, long long T,
                 BatchCtrl* bc, unsigned long long* done, int R, long long spin_limit, int tune,
                 cudaStream_t s);

// host launchers (od_kernels.cu)
int launch_init_ions(const Phys& P, const Bufs& B, cudaStream_t s);
int launch_fpos(const Phys& P, const Bufs& B, int buf, cudaStream_t s);
int launch_pad(const Phys& P, const Bufs& B, cudaStream_t s);
int launch_push_scan(const Phys& P, const Bufs& B, cudaStream_t s);
int launch_forces(const Phys& P, const Bufs& B, const ForceArgs& F, int variant, cudaStream_t s);
int launch_kick(const Phys& P, const Bufs& B, const ForceArgs& F, int mode, cudaStream_t s);
int launch_cp_bump(const Bufs& B, cudaStream_t s);  // advance the close-pair list epoch
// the next step's first INJ_AHEAD injection samples (run beside the pair forces)
int launch_inject_ahead(const Phys& P, const Bufs& B, cudaStream_t s);
// this step's collision velocities (Bufs::coll_v), beside the pair forces
int launch_collide_ahead(const Phys& P, const Bufs& B, cudaStream_t s);
// OML floating charge of every grain into Ctrl::Q (nq Gauss-Legendre nodes glx, glw on [-1, 1])
// E_out at the grain centres into Ctrl::eg (once, at creation)
int launch_grain_eout(const Phys& P, const Bufs& B, cudaStream_t s);
int launch_oml_charge(const Phys& P, const Bufs& B, double n_inf, double m_i, double Z, double T_e, int nq,
                      const double* glx, const double* glw, cudaStream_t s);
int launch_forces_f64(const Phys& P, const Bufs& B, int after_push, cudaStream_t s);
int launch_stats(const Phys& P, const Bufs& B, double* mean_se, cudaStream_t s);
// kind 0: [n][3] -> [3][cap] doubles; 1: [3][cap] -> [n][3]; 2: float4 -> [n][3] doubles;
// 3: [n][3] doubles -> float4
int launch_layout(int kind, const void* src, void* dst, int n, long long cap, cudaStream_t s);
int launch_hist(const Phys& P, const Bufs& B, unsigned long long* counts, int nr, int nz, double inv_dr,
                double inv_dz, int sms, cudaStream_t s);
int launch_eout_grid(double R, double H, double lam, int nx, int nz, int nq, const double* gl_x,
                     const double* gl_w, double* out, cudaStream_t s);

// ion-ion cutoff (od_cut.cu): buffers of the slab sort, tile boxes and tile lists;
// lengths in the pair kernel's scaled units
constexpr int CUT_MAX_TILES = 4096;
struct CutBufs {
    int nslab;
    float zoff, inv_w, rc2_tile, rs2_tile;
    int* bcount;   // [nslab][warps] slab counts
    int* boff;     // their exclusive scan
    int* bsum;     // scan chunk sums
    int* perm;     // sorted position -> ion
    int* rank;     // ion -> sorted position
    float4* fsort; // sorted scaled positions, far dummies after N
    float4* box_lo;
    float4* box_hi;
    int2* units;     // [T (T + 1) / 2] tile pairs (I, J >= I | plain flag) whose boxes meet
    int* n_units;
    int* ucnt;       // [T] tile pairs (J >= I) per tile
    int* ustart;     // [T] first unit of each tile
};
int launch_forces_cut(const Phys& P, const Bufs& B, const ForceArgs& F, const CutBufs& C, int grid, cudaStream_t s);
int launch_cut_dummies(const CutBufs& C, int N, int n_pad, cudaStream_t s);
int cut_blocks_per_sm(int ipt);

// pair-kernel variants: (threads per block, targets per thread, symmetric)
struct ForceVariant {
    int BT, IPT, sym;
};
int num_force_variants();
ForceVariant force_variant(int v);
int force_blocks_per_sm(int variant);

// message returned by od_last_error(NULL) for calls without a handle (od_api.cu)
void set_global_error(const std::string& msg);

int push_tile();  // ions per scan tile
int kick_block(); // threads per block of the kick kernel

}  // namespace od
