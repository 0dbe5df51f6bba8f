/*
 * Oracle for the ion-flow-around-dust time step (OpenDust, arXiv 2205.06557).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded-by-definition
 * FP64 CPU restatement of the method, used to check the CUDA library.  Only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark may load it.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Units are SI throughout.  Section / equation references are to the paper:
 *   Sec. 2            ion model, flow types, boundary, force decomposition
 *   Eq. 1 (Fido)      force on dust from shielded ions plus E_out Q_d
 *   Eq. 2 (Fdd)       dust-dust Coulomb force
 *   Eq. 3 (Fidc)      momentum collected from absorbed ions
 *   Eq. 4 (Fext)      force of the driving field on the dust
 *   App. A            confinement field E_out: cavity potential, 15-term fit, gradient
 *   App. B            flux-conserving re-injection (face fluxes, probabilities, CDFs)
 */
#ifndef OD_ORACLE_H
#define OD_ORACLE_H
#include <stdint.h>

#define ORC_MAX_DUST 8
#define ORC_REC 13   /* q, F_orbit[3], F_dd[3], F_collect[3], F_ext[3] */
#define ORC_EV 13    /* absorbed[8], outflow, injected bottom/top/side, collided */

/* flags */
#define ORC_F_NO_IONION   1   /* drop ion-ion Yukawa forces */
#define ORC_F_NO_EOUT     2   /* drop the confinement field (ions and dust) */
#define ORC_F_NO_BOUNDARY 4   /* no outflow removal, no injection */
#define ORC_F_NO_ABSORB   8   /* dust does not absorb ions */
#define ORC_F_PAPER_SIDE 16   /* side injection without tangential velocity */
#define ORC_F_FLUX_INJECT 32  /* inject a Poisson number of ions per step from the App. B
                                 fluxes instead of replacing each removed ion (N varies) */

#define ORC_Q_GIVEN 0
#define ORC_Q_CONSISTENT 1

typedef struct {
    double x, y, z, a, q0;
} orc_dust;

typedef struct {
    double m_i;        /* ion mass, kg */
    double Z;          /* ion charge number */
    double T_i, T_n, T_e;  /* K */
    double n_inf;      /* ion density far from dust, m^-3 */
    double mach;       /* flow Mach number (c_s = sqrt(Z k T_e / m_i)) */
    double E_ext;      /* driving field along +z, V/m */
    double nu;         /* ion-neutral collision frequency, 1/s */
    double R, H, dt;
    double weight;     /* ions per superion */
    int64_t n_ions;    /* 0 => round(n_inf pi R^2 H / weight) */
    int32_t n_dust;
    int32_t charge_model;
    orc_dust dust[ORC_MAX_DUST];
    uint64_t seed;
    int64_t avg_start; /* first record (1-based step) in the time average */
    int32_t has_alpha; /* 1 => use alpha[] instead of fitting App. A */
    int32_t flags;
    double alpha[15];
    int32_t grid_nx, grid_nz;   /* App. A grid, 0 => 40 */
    int32_t quad_n;             /* Gauss-Legendre points per segment, 0 => 48 */
    int32_t pad_;
    /* ion-ion cutoff (Sec. 5: a switching function that vanishes beyond a fixed
     * distance); r_cut <= 0 => none.  Between r_switch and r_cut the pair energy is
     * multiplied by S(x) = 1 - 10 x^3 + 15 x^4 - 6 x^5, x = (r - r_switch) / (r_cut -
     * r_switch); the force is minus the gradient of the switched energy. */
    double r_cut, r_switch;
} orc_params;

typedef struct orc_state orc_state;

orc_state* orc_create(const orc_params* p, char* err, int errlen);
void orc_destroy(orc_state* s);
int orc_step(orc_state* s, int64_t n);
int64_t orc_num_ions(const orc_state* s);
int64_t orc_step_index(const orc_state* s);
void orc_get_ions(const orc_state* s, double* x, double* v, double* a, uint64_t* id);
int orc_set_ions(orc_state* s, int64_t n, const double* x, const double* v, const uint64_t* id, int64_t next_id);
int orc_load_ions(orc_state* s, int64_t n, const double* x, const double* v, const uint64_t* id, int64_t next_id);
void orc_forces(const orc_state* s, int64_t i0, int64_t i1, double* acc, double* f_orbit);
void orc_derived(const orc_state* s, double* out /* 24 */);
void orc_alpha(const orc_state* s, double* alpha);
void orc_eout(const orc_state* s, double x, double y, double z, double* E);
double orc_cyl_integral(const orc_params* p, double r0, double z0);
void orc_inject_sample(const orc_state* s, uint64_t id, uint32_t step, double* pos, double* vel, int* face);
void orc_records(const orc_state* s, int64_t first, int64_t count, double* rec, int32_t* ev);
void orc_dust_q(const orc_state* s, double* q);
int orc_dust_terms(const orc_state* s, double* mean, double* se);
void orc_philox(const uint32_t key[2], const uint32_t ctr[4], uint32_t out[4]);
/* injected superions of step `step` (1-based) under the flux rule (ORC_F_FLUX_INJECT) */
int64_t orc_injections(const orc_state* s, uint32_t step);
int orc_num_threads(void);

#endif
