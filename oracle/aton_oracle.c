/*
 * aton_oracle.c -- TEST INFRASTRUCTURE: the plain, slow, single-threaded FP64 oracle of one
 * explicit time step of the ATON M1 radiative-transfer method (Aubert & Teyssier 2010).
 *
 * Only the test suite, the smoke check and the CPU-baseline leg of the benchmark load this
 * library. It shares no code with the GPU path. Every function below follows one passage of
 * the paper, cited in its comment, or (where the paper defers to other work) a named
 * publication. The step is taken in the paper's order: transport of (N, F) with the
 * Lax-Friedrichs intercell flux (section 2.2; Appendix Eqs. A1-A3), then the source term,
 * then the chemistry/cooling/absorption operator Phi (Appendix Eq. A4), sub-cycled inside the
 * radiative step (section 2.2, chemistry paragraph).
 *
 * Readings taken where the paper is silent or garbled (all listed in the design notes):
 *  - Eq. 6 prints the two coefficients of the Eddington tensor swapped; the reading used is
 *    D = (1-chi)/2 I + (3chi-1)/2 n(x)n, the only one that gives D = I/3 in the diffusion
 *    limit chi = 1/3 stated beside it.
 *  - chi(f) is the Levermore form (3 + 4f^2) / (5 + 2 sqrt(4 - 3f^2)).
 *  - The Lax-Friedrichs flux is the global one with wave speed c.
 *  - Recombination is case B on the spot; rate fits from Hui & Gnedin (1997) and Cen (1992).
 *  - The chemistry is a backward-difference (creation/destruction) update in the spirit of
 *    Anninos et al. (1997), solved implicitly for (N', y') with y = 1 - x so that the photons
 *    removed from N equal the photo-ionisations exactly.
 *
 * Parity pins of each part are in the test suite; the cooling coefficients are pinned only
 * loosely (published-fit cross-checks), which the design notes record.
 */
#include "aton_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* physical constants, cgs */
static const double ORC_KB = 1.380649e-16;       /* Boltzmann [erg/K] */
static const double ORC_EV = 1.602176634e-12;    /* electron volt [erg] */
static const double ORC_IH_EV = 13.6;            /* H ionisation threshold [eV], section 2.2 */
static const double ORC_T_HI = 157807.0;         /* H ionisation temperature [K] (Hui & Gnedin 1997) */

void orc_default_params(orc_params* p) {
  memset(p, 0, sizeof(*p));
  p->c = 2.99792458e10;
  p->dx = 1.0;
  p->dt = 1.0;
  /* single-group constants of the paper's 50 000 K black body (section 2.2) */
  p->sigma_n = 2.93e-18;
  p->sigma_e = 2.49e-18;
  p->e_gamma_eV = 20.27;
  p->bc = ORC_BC_PERIODIC;
  p->fixed_T = 0;
  p->coll_ion = 1;
  p->cooling = 1;
  p->max_sub = 10000;
  p->T_floor = 1.0;
  p->sub_eps = 0.1;
  p->y_floor = 1e-6;
}

/* ------------------------------------------------------------------------------------------
 * M1 closure. Section 2.2, Eq. 5 (P = D N), Eq. 6 (Eddington tensor, coefficients read as
 * swapped, see header) and the paragraph after it: chi depends only on f = |F|/(cN) and spans
 * 1/3 (diffusion) to 1 (free streaming).
 * ------------------------------------------------------------------------------------------ */
double orc_chi(double f) {
  if (f < 0.0) f = 0.0;
  if (f > 1.0) f = 1.0;
  return (3.0 + 4.0 * f * f) / (5.0 + 2.0 * sqrt(4.0 - 3.0 * f * f));
}

void orc_eddington(double N, double Fx, double Fy, double Fz, double c, double D[9]) {
  double Fv[3] = {Fx, Fy, Fz};
  double Fn = sqrt(Fx * Fx + Fy * Fy + Fz * Fz);
  double f = 0.0;
  if (N > 0.0) f = Fn / (c * N);
  double chi = orc_chi(f);
  double iso = 0.5 * (1.0 - chi);        /* coefficient of I */
  double dir = 0.5 * (3.0 * chi - 1.0);  /* coefficient of n(x)n */
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double nn = 0.0;
      if (Fn > 0.0) nn = (Fv[a] / Fn) * (Fv[b] / Fn);
      D[3 * a + b] = (a == b ? iso : 0.0) + dir * nn;
    }
}

/* ------------------------------------------------------------------------------------------
 * Rate coefficients. The paper defers the chemistry and cooling rates to Anninos et al. (1997)
 * and Cen (1992) (section 2.2, chemistry paragraph). These are the published fits used here.
 * ------------------------------------------------------------------------------------------ */

/* Case-B H recombination rate [cm^3 s^-1], Hui & Gnedin (1997) fit, lambda = 2 T_HI / T. */
double orc_alpha_B(double T) {
  double lam = 2.0 * ORC_T_HI / T;
  return 2.753e-14 * pow(lam, 1.5) / pow(1.0 + pow(lam / 2.740, 0.407), 2.242);
}

/* Collisional ionisation rate of HI by electrons [cm^3 s^-1], Hui & Gnedin (1997) fit. */
double orc_beta_coll(double T) {
  double lam = 2.0 * ORC_T_HI / T;
  return 21.11 * pow(T, -1.5) * exp(-lam / 2.0) * pow(lam, -1.089) /
         pow(1.0 + pow(lam / 0.354, 0.874), 1.101);
}

/* Case-B recombination cooling coefficient [erg cm^3 s^-1] (times n_e n_HII), Hui & Gnedin (1997). */
double orc_cool_rec_B(double T) {
  double lam = 2.0 * ORC_T_HI / T;
  return 3.435e-30 * T * pow(lam, 1.970) / pow(1.0 + pow(lam / 2.250, 0.376), 3.720);
}

/* Collisional excitation cooling of HI [erg cm^3 s^-1] (times n_e n_HI), Cen (1992). */
double orc_cool_coll_exc(double T) {
  return 7.5e-19 * exp(-118348.0 / T) / (1.0 + sqrt(T / 1e5));
}

/* Bremsstrahlung [erg cm^3 s^-1] (times n_e n_HII), Cen (1992) with its Gaunt factor. */
double orc_cool_brems(double T) {
  double l = log10(T) - 5.5;
  double gff = 1.1 + 0.34 * exp(-l * l / 3.0);
  return 1.42e-27 * gff * sqrt(T);
}

/* Net radiative cooling of an H-only gas [erg cm^-3 s^-1] at (T, x, nH). */
double orc_cooling_rate(const orc_params* p, double T, double x, double nH) {
  if (!p->cooling) return 0.0;
  double ne = x * nH, nHII = x * nH, nHI = (1.0 - x) * nH;
  double CR = 1.0;
  if (p->clump_R_A > 0.0) { CR = p->clump_R_A * pow(nH, p->clump_R_b); if (CR < 1.0) CR = 1.0; }
  double L = CR * orc_cool_rec_B(T) * ne * nHII;
  L += orc_cool_coll_exc(T) * ne * nHI;
  if (p->coll_ion) L += ORC_KB * ORC_T_HI * orc_beta_coll(T) * ne * nHI;
  L += orc_cool_brems(T) * ne * nHII;
  return L;
}

/* Heat deposited per photo-ionisation [erg]: the energy absorbed per unit time is
 * c sigma_e N e and the ionisations per unit time are c sigma_n N (section 2.2, the
 * single-group cross-sections), less the 13.6 eV spent on each ionisation. */
double orc_heat_per_ionisation(const orc_params* p) {
  return (p->sigma_e * p->e_gamma_eV - p->sigma_n * ORC_IH_EV) / p->sigma_n * ORC_EV;
}

/* ------------------------------------------------------------------------------------------
 * Transport. Section 2.2 Eqs. 3-4 (moment equations) with Eq. 5 (P = D N) solved by the
 * explicit finite-volume update of Appendix Eq. A2, ũ_i = u_i - dt/dx (F*_{i+1/2} -
 * F*_{i-1/2}), extended to 3-D as in Appendix Eq. A5, with the Lax-Friedrichs intercell flux
 * (section 2.2, last paragraph on the flux): F* = (Phi(u_L) + Phi(u_R))/2 - c (u_R - u_L)/2.
 * Boundaries: periodic, or transmissive (zero-gradient ghost = copy of the boundary cell)
 * with the outward photon flux tallied as escaped.
 * ------------------------------------------------------------------------------------------ */

/* physical flux along axis d of u = (N, Fx, Fy, Fz): (F_d, c^2 N D_{x d}, c^2 N D_{y d}, c^2 N D_{z d}) */
static void orc_phys_flux(int d, const double u[4], double c, double out[4]) {
  double D[9];
  orc_eddington(u[0], u[1], u[2], u[3], c, D);
  out[0] = u[1 + d];
  for (int a = 0; a < 3; ++a) out[1 + a] = c * c * u[0] * D[3 * a + d];
}

static void orc_lf_flux(int d, const double uL[4], const double uR[4], double c, double out[4]) {
  double fL[4], fR[4];
  orc_phys_flux(d, uL, c, fL);
  orc_phys_flux(d, uR, c, fR);
  for (int q = 0; q < 4; ++q) out[q] = 0.5 * (fL[q] + fR[q]) - 0.5 * c * (uR[q] - uL[q]);
}

/* The HLL variant (section 2.2 names it beside LF): the wave speeds are the extreme eigenvalues
 * of the Jacobian of the flux along d, G_d(u) = (F_d, c^2 N D_{x d}, c^2 N D_{y d}, c^2 N D_{z d}).
 * With f = |F|/(cN), mu = F_d/|F| and the closure chi(f), its characteristic polynomial
 * factors into the transverse root c (3 chi - 1) mu / (2 f) (twice) and the quadratic
 * (lambda/c)^2 - chi' mu (lambda/c) + C/4 = 0, so
 *   lambda/c = (chi' mu +- sqrt((chi' mu)^2 - C)) / 2,
 *   C = (1 - mu^2)((3 chi - 1) chi'/f - 2) + 2 chi (1 - 3 mu^2) + 2 chi' f (3 mu^2 - 1),
 * which bound the transverse pair. chi' is differentiated from the Levermore form in closed
 * form here; at f = 0 (or N <= 0) the speeds are -+c/sqrt(3). */
void orc_m1_speeds(const double u[4], double c, int d, double* lo, double* hi) {
  const double N = u[0];
  const double Fn = sqrt(u[1] * u[1] + u[2] * u[2] + u[3] * u[3]);
  double f = (N > 0.0) ? Fn / (c * N) : 0.0;
  if (f > 1.0) f = 1.0;
  const double mu = (Fn > 0.0 && N > 0.0) ? u[1 + d] / Fn : 0.0;
  const double s = sqrt(4.0 - 3.0 * f * f);
  const double chi = (3.0 + 4.0 * f * f) / (5.0 + 2.0 * s);
  /* d chi / d f = [8 f (5 + 2 s) + 6 f (3 + 4 f^2) / s] / (5 + 2 s)^2 */
  const double dchi_over_f = (8.0 * (5.0 + 2.0 * s) + 6.0 * (3.0 + 4.0 * f * f) / s) /
                             ((5.0 + 2.0 * s) * (5.0 + 2.0 * s));
  const double three_chi_m1 = 3.0 * chi - 1.0;
  const double C = (1.0 - mu * mu) * (three_chi_m1 * dchi_over_f - 2.0) +
                   2.0 * chi * (1.0 - 3.0 * mu * mu) + 2.0 * dchi_over_f * f * f * (3.0 * mu * mu - 1.0);
  const double b = dchi_over_f * f * mu;   /* chi' mu */
  double disc = b * b - C;
  if (disc < 0.0) disc = 0.0;
  *lo = 0.5 * c * (b - sqrt(disc));
  *hi = 0.5 * c * (b + sqrt(disc));
}

static void orc_hll_flux(int d, const double uL[4], const double uR[4], double c, double out[4]) {
  double fL[4], fR[4], loL, hiL, loR, hiR;
  orc_phys_flux(d, uL, c, fL);
  orc_phys_flux(d, uR, c, fR);
  orc_m1_speeds(uL, c, d, &loL, &hiL);
  orc_m1_speeds(uR, c, d, &loR, &hiR);
  double lm = loL < loR ? loL : loR;
  double lp = hiL > hiR ? hiL : hiR;
  if (lm > 0.0) lm = 0.0;
  if (lp < 0.0) lp = 0.0;
  if (lp - lm <= 0.0) {   /* both cells stream along the face: their fluxes along d vanish */
    for (int q = 0; q < 4; ++q) out[q] = 0.5 * (fL[q] + fR[q]);
    return;
  }
  for (int q = 0; q < 4; ++q)
    out[q] = (lp * fL[q] - lm * fR[q] + lp * lm * (uR[q] - uL[q])) / (lp - lm);
}

/* neighbour index along d (step s = +1/-1) under the boundary condition; -1 marks "ghost of self" */
static int64_t orc_nb(const orc_params* p, int nx, int ny, int nz, int i, int j, int k, int d, int s) {
  int n[3] = {nx, ny, nz};
  int q[3] = {i, j, k};
  q[d] += s;
  if (q[d] < 0 || q[d] >= n[d]) {
    if (p->bc == ORC_BC_PERIODIC) q[d] = (q[d] + n[d]) % n[d];
    else return -1;
  }
  return (int64_t)q[0] + (int64_t)nx * ((int64_t)q[1] + (int64_t)ny * q[2]);
}

void orc_transport(const orc_params* p, int nx, int ny, int nz,
                   const double* N, const double* Fx, const double* Fy, const double* Fz,
                   double* No, double* Fxo, double* Fyo, double* Fzo, double* escaped) {
  const double c = p->c, lam = p->dt / p->dx, face_dt = p->dx * p->dx * p->dt;
  double esc = 0.0;
#ifdef _OPENMP
#pragma omp parallel for collapse(2) reduction(+ : esc) schedule(static)
#endif
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int64_t id = (int64_t)i + (int64_t)nx * ((int64_t)j + (int64_t)ny * k);
        double u[4] = {N[id], Fx[id], Fy[id], Fz[id]};
        double acc[4] = {0, 0, 0, 0};
        for (int d = 0; d < 3; ++d) {
          int64_t ip = orc_nb(p, nx, ny, nz, i, j, k, d, +1);
          int64_t im = orc_nb(p, nx, ny, nz, i, j, k, d, -1);
          double up[4], um[4];
          for (int q = 0; q < 4; ++q) { up[q] = u[q]; um[q] = u[q]; }
          if (ip >= 0) { up[0] = N[ip]; up[1] = Fx[ip]; up[2] = Fy[ip]; up[3] = Fz[ip]; }
          if (im >= 0) { um[0] = N[im]; um[1] = Fx[im]; um[2] = Fy[im]; um[3] = Fz[im]; }
          double fp[4], fm[4];
          if (p->flux == ORC_FLUX_HLL) {
            orc_hll_flux(d, u, up, c, fp);
            orc_hll_flux(d, um, u, c, fm);
          } else {
            orc_lf_flux(d, u, up, c, fp);   /* face i+1/2 */
            orc_lf_flux(d, um, u, c, fm);   /* face i-1/2 */
          }
          for (int q = 0; q < 4; ++q) acc[q] += fp[q] - fm[q];
          if (ip < 0) esc += fp[0] * face_dt;   /* outward through the high face */
          if (im < 0) esc -= fm[0] * face_dt;   /* outward through the low face */
        }
        No[id] = u[0] - lam * acc[0];
        Fxo[id] = u[1] - lam * acc[1];
        Fyo[id] = u[2] - lam * acc[2];
        Fzo[id] = u[3] - lam * acc[3];
      }
  if (escaped) *escaped += esc;
}

/* ------------------------------------------------------------------------------------------
 * Chemistry, cooling and absorption: the operator Phi of Appendix Eq. A4 on one cell.
 * Section 2.2 (chemistry paragraph): hydrogen only, explicit sub-cycling inside the radiative
 * step "in the spirit of Anninos et al. (1997)"; absorption -kappa N, -kappa F of Eqs. 3-4;
 * the ionisation balance of section 3.2.1 Eq. 14, -nH dx/dt = alpha nH^2 x^2 - (1-x) nH Gamma, written for
 * y = 1 - x, with Gamma = c sigma_n N and case-B alpha, plus collisional ionisation.
 *
 * Each sub-step h takes the backward-difference (creation/destruction) form of Anninos et al.
 * for y and the implicit absorption of the photons, solved together:
 *     y' - y = h [ C_R alpha nH (1-y')^2 - C_I c sigma_n N' y' - beta nH x y' ]
 *     N' - N = -nH C_I c sigma_n h N' y'      (photons removed = photo-ionisations)
 * Eliminating N' = N / (1 + nH k y') (k = C_I c sigma_n h) leaves g(y') = 0 with g concave and
 * increasing on [0, 1], g(0) <= 0 <= g(1); Newton's method from y converges to the root.
 * F decays by the same factor as N. The energy E = 1.5 nH (1+x) kB T gains the photo-heating
 * of the absorbed photons and loses the cooling rate linearised in T (semi-implicit).
 * The sub-step is the largest h <= remaining time with |dy/dt| h <= eps max(y, y_floor) and
 * (heating + cooling) h <= eps E (the heating and the cooling time each bound the step, as
 * their difference cancels near thermal balance), evaluated at the start of the sub-step; the
 * temperature condition is dropped for gas at the floor that would cool (T cannot fall).
 * ------------------------------------------------------------------------------------------ */
int orc_chem_cell(const orc_params* p, double nH, double* N, double* Fx, double* Fy, double* Fz,
                  double* x, double* T, double* absorbed_per_volume, int64_t* nsub) {
  double y = 1.0 - *x;
  if (y < 0.0) y = 0.0;
  if (y > 1.0) y = 1.0;
  double Nc = *N, Tc = *T, fx = *Fx, fy = *Fy, fz = *Fz;
  const double n = nH;
  const double eheat = orc_heat_per_ionisation(p);
  double CR = 1.0, CI = 1.0;
  if (p->clump_R_A > 0.0) { CR = p->clump_R_A * pow(n, p->clump_R_b); if (CR < 1.0) CR = 1.0; }
  if (p->clump_I_A > 0.0) { CI = p->clump_I_A * pow(n, p->clump_I_b); if (CI < 1.0) CI = 1.0; }
  double rem = p->dt;
  double absorbed = 0.0;
  int64_t ns = 0;
  int err = 0;
  while (rem > 0.0) {
    if (ns >= p->max_sub) { err = 1; break; }
    double xi = 1.0 - y;
    double alpha = CR * orc_alpha_B(Tc);
    double beta = p->coll_ion ? orc_beta_coll(Tc) : 0.0;
    double Gam = CI * p->c * p->sigma_n * Nc;
    double dydt = alpha * n * xi * xi - (Gam + beta * n * xi) * y;
    double h = rem;
    double ymax = y > p->y_floor ? y : p->y_floor;
    if (fabs(dydt) * h > p->sub_eps * ymax) h = p->sub_eps * ymax / fabs(dydt);
    double Lam = 0.0;
    if (!p->fixed_T) {
      Lam = orc_cooling_rate(p, Tc, xi, n);
      double heat_rate = n * Gam * y * eheat;                 /* erg cm^-3 s^-1 */
      /* gross rate of change of T: heating and cooling each bounded (heating and cooling
       * times), not their difference, which cancels near thermal balance */
      double rate = (heat_rate + Lam) / (1.5 * ORC_KB * n * (1.0 + xi));
      /* at the floor, cooling cannot lower T: the temperature criterion does not apply */
      int pinned = Tc <= p->T_floor && heat_rate < Lam;
      if (!pinned && rate * h > p->sub_eps * Tc) h = p->sub_eps * Tc / rate;
    }
    /* implicit (N', y') */
    double a = h * alpha * n;
    double b = h * beta * n * xi;
    double kk = CI * p->c * p->sigma_n * h;
    double m = n * kk;
    double Y = y;
    for (int it = 0; it < 200; ++it) {
      double den = 1.0 + m * Y;
      double g = Y - y - a * (1.0 - Y) * (1.0 - Y) + kk * Nc * Y / den + b * Y;
      double gp = 1.0 + 2.0 * a * (1.0 - Y) + kk * Nc / (den * den) + b;
      double Yn = Y - g / gp;
      if (Yn < 0.0) Yn = 0.0;
      if (Yn > 1.0) Yn = 1.0;
      double dY = fabs(Yn - Y);
      Y = Yn;
      if (dY <= 1e-15 * Y) break;
    }
    double fac = 1.0 / (1.0 + m * Y);
    double Nn = Nc * fac;
    double dN = Nc - Nn;                 /* photons absorbed per volume = photo-ionisations */
    absorbed += dN;
    double xn = 1.0 - Y;
    if (!p->fixed_T) {
      double e_old = 1.5 * ORC_KB * n * (1.0 + xi) * Tc;
      double heat = dN * eheat;
      double Tn = (e_old + heat) / (1.5 * ORC_KB * n * (1.0 + xn) + h * Lam / Tc);
      if (Tn < p->T_floor) Tn = p->T_floor;
      Tc = Tn;
    }
    Nc = Nn;
    fx *= fac; fy *= fac; fz *= fac;
    y = Y;
    if (h >= rem) rem = 0.0; else rem -= h;
    ++ns;
  }
  *N = Nc; *Fx = fx; *Fy = fy; *Fz = fz;
  *x = 1.0 - y;
  *T = Tc;
  if (absorbed_per_volume) *absorbed_per_volume += absorbed;
  if (nsub) *nsub = ns;
  return err;
}

/* ------------------------------------------------------------------------------------------
 * One radiative step in the paper's order (Appendix Eqs. A2 and A4; section 2.3 for the
 * sources, which act as per-cell emission with nearest-grid-point assignment):
 *   1. transport of (N, F) from the old state, escaped tally;
 *   2. realisability: N >= 0 (removed amount tallied as clipped), |F| <= c N;
 *   3. sources: N += Ndot dt / V per source, emitted += Ndot dt;
 *   4. Phi per cell, absorbed tally.
 * Budget identity: stored_0 + emitted = stored + absorbed + escaped + clipped.
 * ------------------------------------------------------------------------------------------ */
int orc_step(const orc_params* p, int nx, int ny, int nz,
             double* N, double* Fx, double* Fy, double* Fz, double* x, double* T,
             const double* nH, int64_t nsrc, const int64_t* src_idx, const double* src_rate,
             orc_budget* budget, orc_stats* stats) {
  const int64_t nc = (int64_t)nx * ny * nz;
  const double V = p->dx * p->dx * p->dx;
  double* No = (double*)malloc(sizeof(double) * nc * 4);
  if (!No) return -2;
  double* Fxo = No + nc;
  double* Fyo = No + 2 * nc;
  double* Fzo = No + 3 * nc;
  double esc = 0.0;
  orc_transport(p, nx, ny, nz, N, Fx, Fy, Fz, No, Fxo, Fyo, Fzo, &esc);

  double clipped = 0.0;
#ifdef _OPENMP
#pragma omp parallel for reduction(+ : clipped) schedule(static)
#endif
  for (int64_t id = 0; id < nc; ++id) {
    if (No[id] < 0.0) {
      clipped += No[id] * V;
      No[id] = 0.0; Fxo[id] = 0.0; Fyo[id] = 0.0; Fzo[id] = 0.0;
    } else {
      double Fn = sqrt(Fxo[id] * Fxo[id] + Fyo[id] * Fyo[id] + Fzo[id] * Fzo[id]);
      double lim = p->c * No[id];
      if (Fn > lim) {
        double s = lim / Fn;
        Fxo[id] *= s; Fyo[id] *= s; Fzo[id] *= s;
      }
    }
  }

  double emitted = 0.0;
  for (int64_t s = 0; s < nsrc; ++s) {
    No[src_idx[s]] += src_rate[s] * p->dt / V;
    emitted += src_rate[s] * p->dt;
  }

  double absorbed = 0.0;
  int64_t tot = 0, mx = 0, errc = 0;
#ifdef _OPENMP
#pragma omp parallel for reduction(+ : absorbed, tot, errc) reduction(max : mx) schedule(dynamic, 4096)
#endif
  for (int64_t id = 0; id < nc; ++id) {
    double a = 0.0;
    int64_t ns = 0;
    double xx = x[id], TT = T[id];
    int e = orc_chem_cell(p, nH[id], &No[id], &Fxo[id], &Fyo[id], &Fzo[id], &xx, &TT, &a, &ns);
    x[id] = xx; T[id] = TT;
    absorbed += a * V;
    tot += ns;
    if (ns > mx) mx = ns;
    errc += e;
  }
  memcpy(N, No, sizeof(double) * nc);
  memcpy(Fx, Fxo, sizeof(double) * nc);
  memcpy(Fy, Fyo, sizeof(double) * nc);
  memcpy(Fz, Fzo, sizeof(double) * nc);
  free(No);
  if (budget) {
    budget->emitted += emitted;
    budget->absorbed += absorbed;
    budget->escaped += esc;
    budget->clipped += clipped;
  }
  if (stats) {
    stats->substeps_total += tot;
    if (mx > stats->substeps_max) stats->substeps_max = mx;
    stats->error_cells += errc;
  }
  return errc > 0 ? 1 : 0;
}

int orc_run(const orc_params* p, int nx, int ny, int nz, int nsteps,
            double* N, double* Fx, double* Fy, double* Fz, double* x, double* T,
            const double* nH, int64_t nsrc, const int64_t* src_idx, const double* src_rate,
            orc_budget* budget, orc_stats* stats) {
  int rc = 0;
  for (int s = 0; s < nsteps; ++s) {
    int r = orc_step(p, nx, ny, nz, N, Fx, Fy, Fz, x, T, nH, nsrc, src_idx, src_rate, budget, stats);
    if (r < 0) return r;
    rc |= r;
  }
  return rc;
}

double orc_stored(const orc_params* p, int64_t ncell, const double* N) {
  const double V = p->dx * p->dx * p->dx;
  double s = 0.0;
  for (int64_t i = 0; i < ncell; ++i) s += N[i] * V;
  return s;
}

/* ------------------------------------------------------------------------------------------
 * The same step for one cell from its 3x3x3 neighbourhood (used to check sampled cells of
 * grids too large for a whole-grid oracle run): transport of the centre with the
 * Lax-Friedrichs flux (Appendix Eq. A2 in 3-D), clamp, source, operator Phi (Eq. A4).
 * ------------------------------------------------------------------------------------------ */
int orc_cell_step(const orc_params* p, const double* N27, const double* Fx27, const double* Fy27,
                  const double* Fz27, double x, double T, double nH, double src_rate, double out[7]) {
  const double c = p->c, lam = p->dt / p->dx, V = p->dx * p->dx * p->dx;
  const int ctr = 13;
  const int step[3] = {1, 3, 9};
  double u[4] = {N27[ctr], Fx27[ctr], Fy27[ctr], Fz27[ctr]};
  double acc[4] = {0, 0, 0, 0};
  for (int d = 0; d < 3; ++d) {
    int ip = ctr + step[d], im = ctr - step[d];
    double up[4] = {N27[ip], Fx27[ip], Fy27[ip], Fz27[ip]};
    double um[4] = {N27[im], Fx27[im], Fy27[im], Fz27[im]};
    double fp[4], fm[4];
    if (p->flux == ORC_FLUX_HLL) {
      orc_hll_flux(d, u, up, c, fp);
      orc_hll_flux(d, um, u, c, fm);
    } else {
      orc_lf_flux(d, u, up, c, fp);
      orc_lf_flux(d, um, u, c, fm);
    }
    for (int q = 0; q < 4; ++q) acc[q] += fp[q] - fm[q];
  }
  double N = u[0] - lam * acc[0], Fx = u[1] - lam * acc[1], Fy = u[2] - lam * acc[2],
         Fz = u[3] - lam * acc[3];
  if (N < 0.0) {
    N = 0.0; Fx = 0.0; Fy = 0.0; Fz = 0.0;
  } else {
    double Fn = sqrt(Fx * Fx + Fy * Fy + Fz * Fz);
    if (Fn > c * N) { double s = c * N / Fn; Fx *= s; Fy *= s; Fz *= s; }
  }
  N += src_rate * p->dt / V;
  double ab = 0.0;
  int64_t ns = 0;
  int e = orc_chem_cell(p, nH, &N, &Fx, &Fy, &Fz, &x, &T, &ab, &ns);
  out[0] = N; out[1] = Fx; out[2] = Fy; out[3] = Fz; out[4] = x; out[5] = T; out[6] = ab;
  return e;
}
