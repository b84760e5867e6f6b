/*
 * aton_oracle.h -- TEST INFRASTRUCTURE. Interface of the plain FP64 CPU oracle of one explicit
 * time step of the ATON radiative-transfer method (Aubert & Teyssier 2010, section 2.2 and
 * Appendix A). Only the test suite, the smoke check and the CPU-baseline leg of the benchmark
 * load this library. The GPU product path never links, loads or calls it, and it shares no
 * code, header or constant table with the GPU path.
 *
 * Units are cgs throughout. Arrays are C-order with x fastest: idx = i + nx*(j + ny*k).
 * F is the physical radiative flux [photons cm^-2 s^-1]; N is the photon number density
 * [photons cm^-3]; x is the ionised fraction; T the gas temperature [K]; nH the hydrogen
 * number density [cm^-3].
 */
#ifndef ATON_ORACLE_H
#define ATON_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BC_PERIODIC = 0, ORC_BC_TRANSMISSIVE = 1 };

typedef struct {
  double c;            /* speed of light used by the transport [cm/s] */
  double dx;           /* cell size [cm] */
  double dt;           /* radiative time step [s] */
  double sigma_n;      /* number-averaged H photo-ionisation cross-section [cm^2] */
  double sigma_e;      /* energy-averaged cross-section [cm^2] */
  double e_gamma_eV;   /* mean ionising photon energy [eV] */
  int bc;              /* ORC_BC_* */
  int fixed_T;         /* 1: temperature is held fixed */
  int coll_ion;        /* 1: collisional ionisation (and its cooling) on */
  int cooling;         /* 1: radiative cooling on */
  int max_sub;         /* sub-cycle cap per radiative step */
  double T_floor;      /* temperature floor [K] */
  double sub_eps;      /* sub-step fraction: allowed relative change of y and T per sub-step */
  double y_floor;      /* floor of y in the sub-step criterion */
  double clump_R_A, clump_R_b;  /* recombination clumping C_R = max(1, A nH^b); A=0: C_R = 1 */
  double clump_I_A, clump_I_b;  /* photo-ionisation clumping C_I = max(1, A nH^b); A=0: C_I = 1 */
  int flux;            /* ORC_FLUX_GLF (Lax-Friedrichs, speed c) or ORC_FLUX_HLL */
} orc_params;

#define ORC_FLUX_GLF 0
#define ORC_FLUX_HLL 1

/* Photon-budget accumulators [photons]; "stored" is computed on demand. */
typedef struct {
  double emitted, absorbed, escaped, clipped;
} orc_budget;

typedef struct {
  int64_t substeps_total;  /* sum over cells of chemistry sub-steps taken */
  int64_t substeps_max;    /* largest sub-step count of any cell */
  int64_t error_cells;     /* cells that hit the sub-cycle cap */
} orc_stats;

void orc_default_params(orc_params* p);

/* --- closure (section 2.2, Eqs. 5-6 and the chi paragraph) --- */
double orc_chi(double f);
/* extreme eigenvalues of the M1 flux Jacobian along axis d (0, 1, 2) for u = (N, Fx, Fy, Fz) */
void orc_m1_speeds(const double u[4], double c, int d, double* lo, double* hi);
void orc_eddington(double N, double Fx, double Fy, double Fz, double c, double D[9]);

/* --- rates (fits from the literature the paper defers to; see the .c file) --- */
double orc_alpha_B(double T);
double orc_beta_coll(double T);
double orc_cool_rec_B(double T);
double orc_cool_coll_exc(double T);
double orc_cool_brems(double T);
double orc_cooling_rate(const orc_params* p, double T, double x, double nH);
double orc_heat_per_ionisation(const orc_params* p);

/* --- transport (Appendix Eqs. A1-A3 with the Lax-Friedrichs flux of section 2.2) --- */
void orc_transport(const orc_params* p, int nx, int ny, int nz,
                   const double* N, const double* Fx, const double* Fy, const double* Fz,
                   double* No, double* Fxo, double* Fyo, double* Fzo, double* escaped);

/* --- chemistry operator Phi of Appendix Eq. A4 applied to one cell --- */
int orc_chem_cell(const orc_params* p, double nH, double* N, double* Fx, double* Fy, double* Fz,
                  double* x, double* T, double* absorbed_per_volume, int64_t* nsub);

/* --- one full step: transport, clamp, sources, chemistry, budget --- */
int orc_step(const orc_params* p, int nx, int ny, int nz,
             double* N, double* Fx, double* Fy, double* Fz, double* x, double* T,
             const double* nH, int64_t nsrc, const int64_t* src_idx, const double* src_rate,
             orc_budget* budget, orc_stats* stats);

int orc_run(const orc_params* p, int nx, int ny, int nz, int nsteps,
            double* N, double* Fx, double* Fy, double* Fz, double* x, double* T,
            const double* nH, int64_t nsrc, const int64_t* src_idx, const double* src_rate,
            orc_budget* budget, orc_stats* stats);

double orc_stored(const orc_params* p, int64_t ncell, const double* N);

/* One full step of the centre cell of a 3x3x3 neighbourhood (index 13 = centre, x fastest),
 * whose ghost values the caller has already filled by the boundary rule: transport, clamp,
 * source Ndot (photons/s) and chemistry. out = {N, Fx, Fy, Fz, x, T, absorbed per volume}. */
int orc_cell_step(const orc_params* p, const double* N27, const double* Fx27, const double* Fy27,
                  const double* Fz27, double x, double T, double nH, double src_rate, double out[7]);

#ifdef __cplusplus
}
#endif
#endif
