/*
 * opendust.h -- C ABI of the GB300 (sm_103a) ion-flow-around-dust library.
 *
 * The library advances the paper's method (OpenDust, arXiv 2205.06557) on one GPU:
 * superions in a cylinder of radius R and height H (origin on the axis at mid
 * height, flow along +z; Sec. 2) interact by Yukawa forces screened with the
 * electron Debye length; grains act on ions by bare Coulomb forces and feel the
 * screened ion field (Eq. 1); the ions outside the domain act through the cavity
 * field E_out (App. A); ions move by velocity Verlet in the driving field and
 * collide with neutrals at a constant frequency (Andersen thermostat, Sec. 2);
 * ions that leave the domain or hit a grain are replaced one for one on the
 * boundary (App. B); absorbed ions charge the grain and transfer momentum (Eq. 3);
 * per-dust force terms (Eqs. 1-4) and charges are accumulated in FP64.
 *
 * Conventions for every call:
 *   - units are SI;
 *   - pointers marked "host" are ordinary CPU memory owned by the caller, read or
 *     written only during the call; the library owns all device memory it allocates;
 *   - return value 0 (OD_OK) on success, a negative OD_E* code otherwise; the text of
 *     the last error is available from od_last_error();
 *   - after any error the handle stays valid for od_destroy() and for reads;
 *   - calls on one handle are not thread-safe; different handles are independent.
 */
#ifndef OPENDUST_H
#define OPENDUST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OD_MAX_DUST 8 /* grains per run */
#define OD_REC 13     /* per-dust record: q, F_orbit[3], F_dd[3], F_collect[3], F_ext[3] */
#define OD_EV 13      /* per-step events: absorbed[8], outflow, injected bottom/top/side, collided */
#define OD_NCOUNT 16  /* cumulative counters, see od_counters() */

/* return codes */
#define OD_OK 0
#define OD_EINVAL (-1)    /* invalid parameter or argument */
#define OD_ENOMEM (-2)    /* device allocation failed */
#define OD_ECUDA (-3)     /* a CUDA call failed (message in od_last_error) */
#define OD_ENAN (-4)      /* a non-finite ion position or velocity was produced */
#define OD_EOVERFLOW (-5) /* more ions than the handle's capacity */
#define OD_ETIMEOUT (-6)  /* a device-side wait hit its iteration limit */
#define OD_ENODEV (-7)    /* no CUDA device */
#define OD_ERANGE (-8)    /* a pair-force partial sum left the fixed-point range of the symmetric
                             kernels (two ions nearly coincide) */

/* od_params.flags */
#define OD_F_NO_IONION 1    /* drop the ion-ion Yukawa forces */
#define OD_F_NO_EOUT 2      /* drop the cavity field E_out (ions and grains) */
#define OD_F_NO_BOUNDARY 4  /* no outflow removal (absorbed ions are still replaced) */
#define OD_F_NO_ABSORB 8    /* grains do not absorb ions */
#define OD_F_PAPER_SIDE 16  /* side injection without the tangential thermal velocity */
#define OD_F_FP32_STATE 32  /* round ion positions and velocities to FP32 after every
                               update (precision study: FP32-only ion state) */
#define OD_F_NO_GRAPH 64    /* launch each step's kernels directly, not as a CUDA graph */
#define OD_F_FP64_PAIRS 256 /* study only: ion-ion pair forces in FP64 (one target per thread,
                                libm exp2/sqrt; ~100x slower) for the precision study of the
                                FP32 kernels; not with the cutoff, od_tune or a batch */
#define OD_F_FLUX_INJECT 128 /* inject a Poisson number of ions per step with the mean
                                n_inf (J_bottom + J_top + J_side) dt / weight of the App. B
                                fluxes, instead of one per removed ion: N varies (within a
                                capacity of 1.25 N0 + 256; beyond it a step reports
                                OD_EOVERFLOW); single runs without the cutoff only */

/* od_params.charge_model (Sec. 2 charging options) */
#define OD_Q_GIVEN 0      /* constant charges q0 */
#define OD_Q_CONSISTENT 1 /* OML electron flux + counted absorbed ions */
#define OD_Q_OML 2        /* constant charges: each grain's isolated-sphere OML floating charge in
                             the run's flow (q0 ignored), see od_oml_charge */

typedef struct od_dust {
    double x, y, z; /* position, m; the grain must lie inside the cylinder */
    double radius;  /* m, > 0 */
    double q0;      /* initial (or constant) charge, C */
} od_dust;

typedef struct od_params {
    double ion_mass;          /* m_i, kg */
    double ion_charge_number; /* Z > 0 (1 for singly charged ions) */
    double T_i, T_n, T_e;     /* ion, neutral, electron temperatures, K; T_n <= 0 => T_n = T_i */
    double n_inf;             /* ion density of the unperturbed plasma, m^-3 (electrons: Z n_inf) */
    double mach;              /* flow speed u = mach * sqrt(Z k T_e / m_i); with nu_in > 0 the
                                 driving field is set to E = m_i nu_in u / (Z e) */
    double E_ext;             /* driving field along +z, V/m (field-driven flow, needs nu_in > 0,
                                 flow speed u = Z e E_ext / (m_i nu_in)); give mach or E_ext */
    double nu_in;             /* ion-neutral collision frequency, 1/s; 0 = collisionless */
    double R, H;              /* cylinder radius and height, m */
    double dt;                /* time step, s */
    double weight;            /* real ions per superion, >= 1 typical */
    int64_t n_ions;           /* superions; 0 => round(n_inf pi R^2 H / weight) */
    int32_t n_dust;           /* 0 .. OD_MAX_DUST */
    int32_t charge_model;     /* OD_Q_GIVEN or OD_Q_CONSISTENT */
    const od_dust* dust;      /* host, n_dust entries, copied by od_create */
    uint64_t seed;            /* Philox4x32-10 key for every random draw */
    int64_t avg_start;        /* first step (1-based) included in the time averages; <= 0 => 1 */
    const double* eout_coeffs;/* host, optional: the 15 alpha of App. A's polynomial, SI; NULL =>
                                 computed by quadrature of the uniform ion fill and least squares */
    int32_t flags;            /* OD_F_* */
    int32_t eout_grid;        /* App. A grid nodes per axis minus one; 0 => 40 */
    void* cuda_stream;        /* cudaStream_t for all work; NULL => a stream owned by the library */
} od_params;

typedef struct od_handle od_handle;

/* Create a run: validate p (no device work if invalid, OD_EINVAL), derive the plasma
 * constants, build E_out (App. A), place the initial ions (uniform in the cylinder
 * outside the grains, shifted-Maxwellian velocities) and compute their initial forces.
 * *out receives the handle, or NULL on error (then od_last_error(NULL) has the text). */
int od_create(const od_params* p, od_handle** out);

/* Advance n >= 0 time steps (the canonical order: half kick and drift; absorption and
 * outflow; compaction and re-injection; forces; half kick; collisions; grain update).
 * Work is queued on the run's stream as replayed CUDA graphs (16 steps per graph while 16
 * or more remain, one step per graph for the rest; captured on first use and again after a
 * configuration change); the call waits for it to read the device error word: OD_ENAN,
 * OD_ETIMEOUT or OD_ECUDA report a failure inside the steps. */
int od_step(od_handle* h, int64_t n);

/* Time averages over steps avg_start..current (Sec. 2 results): q[D] mean charge (C)
 * and F[3 D] mean total force (N) = F_orbit + F_dd + F_collect + F_ext. Host arrays. */
int od_dust_state(od_handle* h, double* q, double* F);

/* Release all device memory and the handle. NULL is a no-op. */
void od_destroy(od_handle* h);

/* ---- extras for tests, benchmarks and restarts ---- */

/* Window means and batch-means standard errors (20 equal batches) of every record
 * entry: mean[D][13], se[D][13] (host; se = NaN with fewer than 20 steps). */
int od_dust_terms(od_handle* h, double* mean, double* se);

/* Per-step records for steps first..first+count-1 (1-based): rec[count][D][13] (q is the
 * charge after that step's update; the force terms use the charges the ions felt during
 * the step) and ev[count][13] event counts. Either pointer may be NULL. Host arrays. */
int od_series(od_handle* h, int64_t first, int64_t count, double* rec, int32_t* ev);

/* Cumulative counters (host int64[16]): absorbed per grain [0..7], outflow [8],
 * injected bottom/top/side [9..11], collided [12], steps [13], ions [14], next id [15]. */
int od_counters(od_handle* h, int64_t* out);

/* Current charges q[D] (C) and the Eq. 1 force on every grain f_orbit[3 D] (N) at the
 * last force evaluation (host). */
int od_dust_now(od_handle* h, double* q, double* f_orbit);

/* Copy the ion state to host arrays: x[3 n], v[3 n] (FP64), a[3 n] (FP32 accelerations
 * of the last force evaluation, as doubles), id[n]. cap is the array length in ions;
 * returns the ion count n (>= 0) or an error; any pointer may be NULL. */
int64_t od_get_ions(od_handle* h, double* x, double* v, double* a, uint64_t* id, int64_t cap);

/* Replace the ion state with n ions from host arrays x[3 n], v[3 n], id[n]; next_id is
 * the id given to the next injected ion. If a (host, 3 n) is NULL the forces and the
 * grain force are recomputed for the new positions; otherwise a is taken as the
 * accelerations (restart from od_get_ions output). n may not exceed the ion count the
 * handle was created with (OD_EOVERFLOW). */
int od_set_ions(od_handle* h, const double* x, const double* v, const double* a, const uint64_t* id,
                int64_t n, uint64_t next_id);

/* Ion-ion cutoff (Sec. 5: a switching function that is zero beyond a fixed cutoff
 * distance, so that the cost grows far slower than N^2 in long domains).  The paper does
 * not give the switching form; here the Yukawa pair energy is multiplied by
 * S(x) = 1 - 10 x^3 + 15 x^4 - 6 x^5, x = (r - r_switch) / (r_cut - r_switch) on
 * [r_switch, r_cut], S = 1 below and 0 above, and the pair force is minus the gradient of
 * the switched energy (continuous, zero at r_cut).  The ion-grain forces, Eq. 1 and
 * E_out are unchanged.  0 <= r_switch < r_cut (m); r_cut <= 0 switches the cutoff off.
 * Every later force evaluation sorts the ions by z and visits only tile pairs whose
 * bounding boxes come within r_cut (suited to the elongated domains of the paper's
 * cutoff study); the call re-evaluates the forces of the current state.  At most
 * 2,097,152 ions; OD_EINVAL when the partial sums would need more than 48 GB (a cutoff
 * long against the domain) or on a batch member; od_tune is not available while the
 * cutoff is on.  Partial-sum slots per ion: the neighbour tiles of a uniform density with
 * a margin, grown to the largest neighbour count of the current positions (plus a quarter)
 * whenever od_set_cutoff, od_set_ions or od_load finds more.  A step whose positions
 * outgrow them skips its ion-ion forces and reports OD_EOVERFLOW; od_load of an earlier
 * checkpoint or od_set_ions then resizes the slots and clears the report. */
int od_set_cutoff(od_handle* h, double r_cut, double r_switch);

/* Checkpoint and restart (the paper's runs last tens of thousands of steps, Sec. 4).
 * od_save writes the whole state of a single run to a binary file: the creation
 * parameters, the E_out coefficients, positions, velocities, ids and accelerations, the
 * control block (step, next id, charges, window sums, counters) and every per-step
 * record so far, plus the pair-kernel choice.  od_load creates a new run from such a
 * file on cuda_stream (NULL: a stream owned by the library); continuing it gives the
 * same results, bit for bit, as continuing the saved run on the same GPU model.  The file
 * is in host byte order and tied to this library's layout: a foreign, truncated or
 * inconsistent file is OD_EINVAL before any device work (then od_last_error(NULL)). */
int od_save(od_handle* h, const char* path);
int od_load(const char* path, void* cuda_stream, od_handle** out);
/* number of grains of a run (>= 0), or a negative error code */
int od_num_dust(od_handle* h);

/* Ion dumps for external viewers (the paper's density pictures, Sec. 4, are made from
 * such files): the current ions as extended XYZ (OD_DUMP_XYZ: count line, a properties
 * line with step and time, then "I x y z vx vy vz id", SI) or CSV (OD_DUMP_CSV:
 * id,x,y,z,vx,vy,vz), full FP64 precision. */
#define OD_DUMP_XYZ 0
#define OD_DUMP_CSV 1
int od_write_ions(od_handle* h, const char* path, int32_t format);

/* Time-averaged ion density n(r, z) on an nr x nz grid over r in [0, R), z in
 * [-H/2, H/2] (the axisymmetric density maps of Sec. 4).  od_density_enable allocates
 * and zeroes the counts (1 <= nr, nz <= 4096, nr nz <= 2^22; 0, 0 switches the map off)
 * and every later od_step adds the ions' end-of-step positions (a binning kernel in the
 * step; bins from FP64 positions with correctly rounded operations, integer counts).
 * od_density_read copies counts[nz][nr] (uint64, host, may be NULL), the density
 * density[nz][nr] = counts w / (samples V_bin) in m^-3 (host, may be NULL; V_bin the
 * annulus volume) and the number of steps accumulated.  Single runs only (not batch
 * members). */
int od_density_enable(od_handle* h, int32_t nr, int32_t nz);
int od_density_read(od_handle* h, uint64_t* counts, double* density, int64_t* samples);

/* Derived constants (host double[32]): lambda_De, c_s, sig_i, sig_n, u, E, q, m, p_bottom,
 * p_top, p_side, T_bottom, T_bottom+top, T_coll, N (the ion count the buffers and kernel
 * plans are sized for: under OD_F_FLUX_INJECT the capacity, and the live count is
 * od_counters()[14]), alpha[0..14] (at 15..29), capacity, SMs. */
int od_info(od_handle* h, double* out);

/* Per-kernel timing (profiling mode): when on, od_step launches kernels directly with
 * CUDA events around each and accumulates their durations, reading the events 64 steps
 * at a time and at the end of the call (the host does not wait between steps, so the
 * device runs them back to back; results are bit-identical to the graph replay).
 * od_set_profiling resets the sums. od_kernel_times: ms[4] and launches[4] for
 * push+scan+inject, pair forces, kick+collide with the grain update (which runs in the
 * kick's last block), and a fourth entry kept at zero time. Host arrays. */
int od_set_profiling(od_handle* h, int on);
int od_kernel_times(od_handle* h, double* ms, int64_t* launches);

/* Pair-kernel autotuner (the all-pairs force evaluation of Sec. 5 is the hot spot).
 * Variants 0-7 evaluate every ordered pair (threads per block x targets per thread:
 * 64x1, 64x2, 128x2, 128x4, 256x2, 256x4, 128x8, 64x8); variants 8-11 evaluate each
 * unordered pair once and apply it to both ions (Newton's third law; 128x2, 128x4,
 * 256x2, 256x4) and variants 12-18 do the same with packed FP32-pair arithmetic (128x2,
 * 128x4, 256x2, 256x4, 128x8, 64x8, 32x8), at the
 * price of one partial-sum slot per tile of BT x IPT ions for every ion (device memory
 * N_pad^2 / (BT IPT) x 16 bytes, allocated by the call that selects the variant).  All
 * give forces within FP32 rounding of each other.
 * od_tune times every variant at four work granularities (4, 8, 16, 32 units per
 * persistent block; the symmetric variants have fixed-size units and are timed at the
 * first only) and three persistent grid sizes (CTAs per SM: the occupancy limit, 4, 2)
 * on the run's current ions, reps launches of the force evaluation plus the kick (which
 * sums the partial slots) each, and writes these averages in ms to ms[n_variants][4][3]
 * (host, may be NULL; -1 where a setting is not timed; symmetric layouts needing more
 * than 1/8 of the free device memory are skipped).  The three fastest settings are then
 * timed again in turn, three rounds of reps launches each, and the fastest in total is
 * kept (one of the three smallest entries of ms).  It then
 * re-evaluates the current state's forces with the chosen kernel and frees unused slot
 * memory.  Without tuning a run uses variant 0 up to 4,096 ions, 2 up to 32,768, then 15
 * while its slots fit in 16 GB (~1.05 million ions), else 3.
 * od_set_force_config applies a known choice (e.g. from a cache; blocks_per_sm 0 =
 * occupancy limit) and od_get_force_config reports the current one and the number of
 * variants.  The ion state is not changed; call between steps. */
int od_tune(od_handle* h, int reps, double* ms, int* best_variant, int* best_units_per_block, int* best_blocks_per_sm);
int od_set_force_config(od_handle* h, int variant, int units_per_block, int blocks_per_sm);
int od_get_force_config(od_handle* h, int* variant, int* units_per_block, int* blocks_per_sm, int* n_variants);

/* Pipe micro-benchmarks of the current GPU (the ALU roofline of the pair kernel), host
 * double[9]: operations per second per SM of FP32 FMA, MUFU rsqrt, MUFU ex2 and FP64 FMA;
 * the latency (ns) of a dependent FP64 FMA and of a dependent FP64 exp; the device's
 * maximum SM clock (MHz); operations per second per SM of MUFU rcp and MUFU lg2.  Divide
 * by the SM clock seen while they ran for per-clock rates.  Each rate comes from 64 warps
 * per SM with eight independent chains each (throughput, not latency); about 10 ms in all. */
int od_measure_peaks(double* out);

/* OML floating charge (C) of an isolated grain of the given radius in the plasma and flow
 * of p (Sec. 2 "oml" option): the ion current of the drifting Maxwellian with the OML
 * cross-section balances the Boltzmann electron current.  Host computation. */
int od_oml_charge(const od_params* p, double radius, double* Q);

/* ---- batches: many independent runs in one launch per step ----
 * The paper's sweeps (Sec. 4: drag versus Mach number, versus collision frequency)
 * are sets of independent runs.  A batch advances R runs of uneven ion count with ONE
 * persistent kernel launch per step (replayed from a CUDA graph): the runs' step phases
 * are tasks taken by a resident grid in dependency order.
 *   od_create_batch   ps[R] (host, copied; ps[0].cuda_stream is used for the batch, the
 *                     other streams are ignored); each run is created as by od_create
 *   od_batch_step     n steps of every run; same error codes as od_step (first failing run)
 *   od_batch_run      the handle of run r, for every read call (od_dust_state, od_series,
 *                     od_counters, od_get_ions, od_info ...); the batch owns it: do not
 *                     destroy it, step it, replace its ions or tune it on its own
 *   od_batch_tune     times every run's pair tasks followed by its kick tiles (accelerations
 *                     only) at targets-per-thread {2,4,8} x source chunk {2048, 4096, 8192,
 *                     0}, where chunk 0 means symmetric tile pairs of 128 x targets-per-
 *                     thread ions (each unordered pair once, packed FP32 pairs, one partial
 *                     slot per tile for every ion); ms[12] (host, may be NULL) gets the
 *                     average ms per launch, [ipt index][chunk index]; keeps the fastest and
 *                     recomputes the accelerations with it; positions, velocities and
 *                     grain state are not changed
 *   od_batch_set_config applies a known choice (targets per thread 2, 4 or 8; chunk 0
 *                     or >= 256); od_destroy_batch
 *                     frees everything
 *   od_batch_last_error text of the last error on b (or of the last failed create). */
typedef struct od_batch od_batch;
int od_create_batch(const od_params* ps, int32_t R, od_batch** out);
int od_batch_step(od_batch* b, int64_t n);
od_handle* od_batch_run(od_batch* b, int32_t r);
int od_batch_size(const od_batch* b);
int od_batch_tune(od_batch* b, int reps, double* ms, int* best_targets_per_thread, int* best_chunk);
int od_batch_set_config(od_batch* b, int targets_per_thread, int chunk);
void od_destroy_batch(od_batch* b);
const char* od_batch_last_error(const od_batch* b);

/* ---- learned warm start for the self-consistent charge (no counterpart in the paper) ----
 * A set-pooled MLP maps (Mach number, collision frequency, T_e/T_i; per grain position and
 * radius) to per-grain (charge, force) in normalised units; its prediction only seeds the
 * charges q0 of a run with the "consistent" model (Sec. 2), and the method itself then
 * converges and judges the result.  Layers: per grain 7 -> 256 -> 256 (relu), masked mean
 * over the sample's grains, [h, mean] 512 -> 256 -> 256 (relu) -> 4.  FP32 master weights
 * with Adam; every product uses BF16 weights and activations with FP32 accumulation on
 * the tensor cores.  Inputs are host arrays: x[B][8][7], mask[B][8] (1 present, 0 absent),
 * targets[B][8][4]; B <= max_batch.  Parameters are flattened layer by layer as W
 * (out x in, row-major, in padded to 16 for the first layer, out padded to 16 for the last)
 * followed by b (out).  stream: cudaStream_t (NULL = legacy default stream). */
typedef struct od_sur od_sur;
int od_sur_create(int max_batch, uint64_t seed, void* stream, od_sur** out);
void od_sur_destroy(od_sur* s);
int od_sur_num_params(const od_sur* s);
int od_sur_get_params(od_sur* s, float* params);
int od_sur_set_params(od_sur* s, const float* params);
int od_sur_forward(od_sur* s, const float* x, const float* mask, int B, float* y);
int od_sur_gradients(od_sur* s, const float* x, const float* mask, const float* targets, int B, double* loss,
                     float* grads);
int od_sur_train_step(od_sur* s, const float* x, const float* mask, const float* targets, int B, float lr,
                      double* loss);
const char* od_sur_last_error(const od_sur* s);

/* Matrix-product engine of the network's forward and backward passes:
 *   OD_GEMM_TCGEN05 (default): the fifth-generation tensor cores (tcgen05.mma, M = 128
 *     tiles, FP32 accumulators in tensor memory, operands staged in shared memory);
 *   OD_GEMM_MMA_SYNC: warp-level mma.sync m16n8k16 tiles, kept as an independent
 *     cross-check of the first.
 * Both take BF16 operands and accumulate in FP32; their results differ only in the order
 * of the FP32 additions.  Returns OD_EINVAL for another value. */
#define OD_GEMM_TCGEN05 0
#define OD_GEMM_MMA_SYNC 1
int od_sur_set_gemm(od_sur* s, int engine);

/* One product with either engine on device buffers (the network's products, exposed for
 * tests): C[M][N] = A[M][K] B[N][K]^T (+ bias[N]) (max(., 0) if relu), FP32 C and,
 * if Cb is not NULL, its BF16 rounding.  A, B: BF16 (bit pattern in uint16), row-major,
 * K contiguous; bias: FP32 or NULL; all device pointers, 16-byte aligned.  Sizes:
 * K and N multiples of 16 for both engines, M a multiple of 16 for OD_GEMM_MMA_SYNC
 * (any M >= 1 for OD_GEMM_TCGEN05).  err: device int the caller zeroes; a tensor-core
 * wait that gives up (never expected) ORs 2 into it, the call still returns.  Asynchronous
 * on `stream` (cudaStream_t, NULL = legacy default stream).  OD_EINVAL for bad sizes or
 * engine, OD_ECUDA for a launch failure. */
int od_gemm_bf16(const uint16_t* A, const uint16_t* B, const float* bias, float* C, uint16_t* Cb, int M, int N,
                 int K, int relu, int engine, int* err, void* stream);

/* Failure-detection self-test (no counterpart in the paper): runs one push/scan kernel in
 * which the first scan tile withholds its prefix, so the look-back wait of the next
 * tile finds no inclusive prefix and gives up after `polls` polls instead of its usual
 * ~4 s limit.  Expected return: OD_ETIMEOUT, with the GPU context still usable.  The
 * run's ion state is left inconsistent: destroy the handle afterwards.  Needs more than
 * 256 ions. */
int od_selftest_wait_timeout(od_handle* h, int64_t polls);

/* Text of the last error on h, or of the last failed call without a handle (od_create,
 * od_pair_accel_static) when h is NULL. */
const char* od_last_error(const od_handle* h);

/* ---- pair forces without device allocation (the paper has no counterpart) ----
 *
 * For callers that cannot allocate device memory: host applications or plugins whose
 * framework owns every device allocation and forbids allocations outside its pool, and
 * latency-critical loops in which a cudaMalloc (which may synchronise the device) is not
 * acceptable.
 *
 * Computes the ion-ion Yukawa accelerations of n ions already in device memory,
 *     a_i = k * sum_{j != i} (1 + r_ij/lambda_De) exp(-r_ij/lambda_De) (x_i - x_j) / r_ij^3,
 * with the same FP32 pair arithmetic as od_step and the same FP64 correction of pairs
 * closer than 0.005 max(1, |s|max / 4) scaled units s = r log2(e) / lambda_De (k = q^2 /
 * (4 pi eps0 m) for superions of charge q and mass m).
 *   x       device, [n][3] FP64 positions (m), read only
 *   n       0 .. OD_STATIC_MAX_IONS (OD_EINVAL beyond)
 *   a       device, [n][3] FP32 accelerations (m/s^2), written
 *   stream  cudaStream_t for the work (NULL = the legacy default stream); the call only
 *           queues work and does not wait for it
 * Scratch: a fixed array inside the library (about 5.1 MiB: scaled positions, 8 partial
 * sums per ion, 65,536 close-pair cell buckets and their links, one bound word) that every
 * GPU loading the library holds until the process exits; no cudaMalloc, cudaFree or
 * allocating library routine is called.  The first call on a device (and the first after
 * its context changes, e.g. after cudaDeviceReset) looks up the array's device address
 * with that device current; make that first call before any stream capture.  Every call
 * shares the one array and leaves its contents behind: the bound word is cleared by each
 * call (cudaMemsetAsync), everything else it reads is written by the same call first.
 * Calls whose work overlaps on the GPU (different streams, or different host threads on
 * one device) race on the array and give wrong results: serialise them. */
#define OD_STATIC_MAX_IONS 32768
int od_pair_accel_static(const double* x, int64_t n, double lambda_De, double k, float* a, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* OPENDUST_H */
