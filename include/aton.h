/*
 * aton.h -- C ABI of the B300 ATON step library (libaton.so).
 *
 * One explicit time step of the ATON method (Aubert & Teyssier 2010): moment transport of a
 * single-group ionising photon field (density N, flux F) with the M1 closure and the
 * Lax-Friedrichs intercell flux (section 2.2, Eqs. 3-7; Appendix Eqs. A1-A3, A5), point-source
 * injection (section 2.3: sources act as per-cell emission, nearest grid point), then the
 * sub-cycled hydrogen photo-chemistry, photo-heating and cooling with photon absorption, the
 * operator Phi of Appendix Eq. A4 (section 2.2, chemistry paragraph; section 3.2.1, Eq. 14).
 *
 * Conventions shared by every entry point:
 *  - Units are cgs at the boundary: N [photons cm^-3], F [photons cm^-2 s^-1], T [K],
 *    nH [cm^-3], rates [photons s^-1], budgets [photons].
 *  - Fields are dense 3-D arrays in C order with x fastest: idx = i + nx*(j + ny*k), float32.
 *  - Every array argument is copied; the library never keeps a caller pointer. `where`
 *    (ATON_HOST / ATON_DEVICE) says whether the pointers are host memory (pageable or pinned)
 *    or device memory on the handle's device.
 *  - The handle owns all device memory it allocates and frees it in aton_finalize.
 *  - Work is queued on the handle's stream. Calls that return data to the host synchronise
 *    that stream; aton_step does not.
 *  - Return 0 on success or a negative ATON_ERR_* code; aton_strerror() describes it and
 *    aton_last_message() gives the detail of the last failure on this thread.
 *  - A handle is not thread-safe; use one handle per host thread. Handles on different devices
 *    may be created and used from different threads at once. A handle lives on the device that
 *    was current at aton_init: make every call on it with that device current.
 */
#ifndef ATON_H
#define ATON_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define ATON_OK 0
#define ATON_ERR_BADARG (-1)    /* invalid argument: size, pointer, index, or dt above the CFL limit */
#define ATON_ERR_NOMEM (-2)     /* device or host allocation failed */
#define ATON_ERR_CUDA (-3)      /* a CUDA runtime/driver call failed (detail in aton_last_message) */
#define ATON_ERR_SUBCYCLE (-4)  /* a cell reached the chemistry sub-cycle cap (state kept, flagged) */
#define ATON_ERR_NONFINITE (-5) /* a non-finite value was produced or supplied */
#define ATON_ERR_STATE (-6)     /* call out of order (e.g. stepping before aton_set_fields) */

/* ---- enumerations ---- */
#define ATON_HOST 0
#define ATON_DEVICE 1
#define ATON_BC_PERIODIC 0
#define ATON_BC_TRANSMISSIVE 1
#define ATON_SRC_REPLACE 0
#define ATON_SRC_APPEND 1
#define ATON_MODE_FUSED 0      /* one fused transport+source+chemistry kernel per step (TMA-staged
                                  planes when nx is a multiple of 4, else plain loads) */
#define ATON_MODE_UNFUSED 1    /* plain three-kernel step (transport; sources; chemistry) */
#define ATON_MODE_FUSED_LDG 2  /* the fused kernel with plain per-thread loads (no TMA) */

/* photon-budget vector returned by aton_photon_budget [photons] */
#define ATON_B_EMITTED 0   /* sum of Ndot dt injected by the sources */
#define ATON_B_STORED 1    /* sum of N V now on the grid */
#define ATON_B_ABSORBED 2  /* photons absorbed by photo-ionisations */
#define ATON_B_ESCAPED 3   /* net photons that left through transmissive faces */
#define ATON_B_CLIPPED 4   /* N removed by the N >= 0 clamp (<= 0: photons added) */
#define ATON_B_STORED0 5   /* sum of N V when the fields were last set */
#define ATON_BUDGET_LEN 6
/* identity: stored0 + emitted = stored + absorbed + escaped + clipped */

typedef struct aton_ctx* aton_handle;
typedef struct aton_mlp* aton_mlp_handle;

/* Physical and numerical parameters. Defaults (aton_default_params) are the paper's single
 * group for a 50 000 K black body (section 2.2: sigma_e 2.49e-18, sigma_n 2.93e-18 cm^2,
 * e 20.27 eV), periodic boundaries, evolving temperature with cooling and collisional
 * ionisation, sub-step fraction 0.1 and a cap of 10 000 sub-steps. */
typedef struct {
  double sigma_n;     /* number-averaged H photo-ionisation cross-section [cm^2] */
  double sigma_e;     /* energy-averaged cross-section [cm^2] */
  double e_gamma_eV;  /* mean ionising photon energy [eV] */
  int bc;             /* ATON_BC_* */
  int fixed_T;        /* nonzero: temperature is not evolved */
  int coll_ion;       /* nonzero: collisional ionisation and its cooling */
  int cooling;        /* nonzero: radiative cooling */
  int max_sub;        /* chemistry sub-cycle cap per radiative step (>= 1) */
  double T_floor;     /* temperature floor [K] (> 0) */
  double sub_eps;     /* allowed relative change of y = 1-x and of T per sub-step (0, 1] */
  double y_floor;     /* floor of y in the sub-step criterion (> 0) */
  double clump_R_A, clump_R_b; /* recombination clumping C_R = max(1, A nH^b); A = 0: off
                                  (section 3.2.1, Eq. 15, read with C_R on the
                                  recombination term and C_I on photo-ionisation) */
  double clump_I_A, clump_I_b; /* photo-ionisation clumping C_I = max(1, A nH^b); A = 0: off */
  int flux;           /* intercell flux: ATON_FLUX_GLF (default) or ATON_FLUX_HLL */
} aton_params;

/* Intercell flux (section 2.2: the code offers Lax-Friedrichs and HLL; the paper uses LF).
 * GLF: face flux (Phi_L + Phi_R)/2 - c (u_R - u_L)/2, wave speed c.
 * HLL: (l+ Phi_L - l- Phi_R + l+ l- (u_R - u_L)) / (l+ - l-) with l- = min(0, lo_L, lo_R),
 * l+ = max(0, hi_L, hi_R), lo/hi the extreme eigenvalues of the M1 flux Jacobian along the face
 * normal in each cell: with chi(f), chi'(f) of the closure and mu the cosine between F and the
 * normal, lo, hi = c (chi' mu -/+ sqrt((chi' mu)^2 - C)) / 2,
 * C = (1 - mu^2)((3 chi - 1) chi' / f - 2) + 2 chi (1 - 3 mu^2) + 2 chi' f (3 mu^2 - 1)
 * (the roots of the Jacobian's characteristic polynomial besides the transverse speed
 * c (3 chi - 1) mu / (2 f); +-c/sqrt(3) at f = 0, c mu at f = 1). HLL runs in the one-launch
 * fused step only in ATON_MODE_FUSED with nx a multiple of 4 (the TMA-staged kernel); with
 * nx not a multiple of 4, and in ATON_MODE_FUSED_LDG, it falls back to the plain three-kernel
 * step, with the same results up to rounding. aton_launches_per_step reports which path a
 * handle takes (1: fused, 3: plain). */
#define ATON_FLUX_GLF 0
#define ATON_FLUX_HLL 1

/* Counters accumulated since aton_set_fields. */
typedef struct {
  int64_t steps;            /* radiative steps taken */
  int64_t substeps_total;   /* chemistry sub-steps summed over cells and steps */
  int64_t substeps_max;     /* largest sub-step count of any cell in any step */
  int64_t error_cells;      /* cell-steps that reached the sub-cycle cap */
  int64_t nonfinite_cells;  /* cell-steps that produced a non-finite value */
  int64_t surrogate_cells;  /* cell-steps whose chemistry the surrogate replaced */
  double max_f;             /* largest reduced flux |F|/(cN) of the current state (cells with
                               N > 1e-30; the M1 closure of section 2.2 needs f <= 1) */
} aton_diag;

/* Chemistry surrogate in the step (see aton_set_surrogate). */
typedef struct {
  int enabled;           /* nonzero: offer cells to the network */
  double gate_substeps;  /* offer a cell when its explicit sub-step estimate is >= this */
  double residual_max;   /* accept a prediction when its photon residual is <= this */
} aton_surrogate_params;

/* Fills *p with the defaults above. Never fails. */
void aton_default_params(aton_params* p);

/* Creates a handle for an nx*ny*nz grid of cubic cells of size dx_cm, speed of light c_cms
 * (a reduced value is allowed) and radiative step dt_s, on the current CUDA device.
 * The explicit scheme needs dt < dx/c (section 2.2, Eq. 7); the unsplit 3-D Lax-Friedrichs
 * update used here is positive only for 3 c dt / dx <= 1, which is enforced.
 * Allocates the device state (double-buffered N, F; y, T, nH) and a stream. The first handle
 * made on a device also sets the kernels' shared-memory limits there (once per device).
 * Errors: BADARG (sizes < 1, cell count above 2^31-1, non-positive dx/c/dt, 3 c dt/dx > 1,
 * out == NULL, a current device index of 64 or more), NOMEM, CUDA. On error *out is set to
 * NULL and everything allocated so far is released. For tests of that clean-up, the
 * environment variable ATON_TEST_FAIL_ALLOC=k makes the k-th of the handle's 15 device
 * allocations (counting from 0) fail with NOMEM without allocating. */
int aton_init(int nx, int ny, int nz, double dx_cm, double c_cms, double dt_s, aton_handle* out);

/* Releases every resource of the handle (NULL is ignored); the caller's current device is kept. */
void aton_finalize(aton_handle h);

/* Replaces the parameters. Validated (BADARG on out-of-range values). Takes effect at the
 * next aton_step. */
int aton_set_params(aton_handle h, const aton_params* p);
int aton_get_params(aton_handle h, aton_params* p);

/* Runs the work of this handle on an existing CUDA stream (cudaStream_t cast to void*; NULL
 * restores the handle's own stream). The caller keeps ownership of the stream and must keep
 * it alive while the handle uses it. */
int aton_set_stream(aton_handle h, void* stream);

/* Chooses the kernel path: ATON_MODE_FUSED (default), ATON_MODE_UNFUSED or
 * ATON_MODE_FUSED_LDG, and the number of steps captured in one CUDA graph (0: no graphs,
 * plain launches). */
int aton_set_exec(aton_handle h, int mode, int graph_batch);
int aton_get_exec(aton_handle h, int* mode, int* graph_batch, int* ty, int* tz);

/* Sets the tile of the fused kernel: ty rows of 32 cells per CTA and tz planes per z-slab.
 * ty in {4, 8, 16}; tz >= 1. */
int aton_set_tile(aton_handle h, int ty, int tz);

/* Rows of the fused tile per thread (1 or 2; default 2). With 2, a CTA of ty/2 warps updates
 * the same 32 x ty tile, each thread two neighbouring rows, which spreads the per-plane work
 * that does not grow with the cells (stage wait, barrier, loop) and the halo rows over more
 * cells. It applies to the TMA-staged kernel at tile heights 8 and 16 with the GLF flux;
 * elsewhere the step runs one row per thread. aton_autotune chooses it with the tile. The
 * fields do not depend on it beyond floating-point contraction (separately compiled kernels). */
int aton_set_tile_rows(aton_handle h, int rows);
int aton_get_tile_rows(aton_handle h, int* rows);

/* Times the fused kernels (TMA-staged where the grid allows it, and plain-load) on a scratch
 * copy of the current state for each candidate tile (and, for the TMA-staged kernel, one or two
 * rows per thread) and keeps the fastest kernel and tile (the
 * simulation state is not advanced; an unfused mode stays unfused). `steps` per candidate
 * (>= 1), then the three fastest once more over 3 x `steps` (short timings are noisy). Writes the chosen (ty, tz) and its time per step [ms] when the pointers are not NULL;
 * aton_get_exec reports the chosen mode. */
int aton_autotune(aton_handle h, int steps, int* ty_out, int* tz_out, float* ms_out);

/* Copies the state in (section 2.2: energy density, flux, temperature, ionisation fraction
 * and baryon density, the per-cell quantities of the Appendix). N, Fx, Fy, Fz, T, nH are
 * required; the ionisation state is given either as the neutral fraction y (preferred:
 * stored as is, no cancellation near full ionisation) or as the ionised fraction x
 * (converted y = 1 - x on the device); exactly one of x, y must be non-NULL.
 * Resets the photon budget and the counters; stored0 becomes sum N V.
 * Errors: BADARG (NULL pointers, both/neither of x,y, bad where), NONFINITE (a non-finite or
 * negative N, T <= 0, nH not a positive normal float (below 1.18e-38), y outside [0,1]:
 * checked on the device), CUDA. */
int aton_set_fields(aton_handle h, const float* N, const float* Fx, const float* Fy,
                    const float* Fz, const float* x, const float* y, const float* T,
                    const float* nH, int where);

/* Copies the current state out. Any output pointer may be NULL (skipped). x and y are the
 * ionised and neutral fractions. Synchronises the stream. Errors: BADARG, STATE, CUDA. */
int aton_get_fields(aton_handle h, float* N, float* Fx, float* Fy, float* Fz, float* x,
                    float* y, float* T, int where);

/* Sets (REPLACE) or extends (APPEND) the point-source list: cell_idx[s] in [0, ncell) (linear
 * index as above), rate_per_s[s] >= 0 photons/s. Host arrays, read before the call returns
 * (the caller may reuse them at once; the device copy is queued on the handle's stream without
 * waiting for a running step). Sources in the same cell are summed, in the order given after
 * any existing entry. Each step adds rate*dt/V to N of its cell after transport and before
 * chemistry (section 2.3 nearest-grid-point emission; S in Eq. 3 and Appendix Eq. A2).
 * Errors: BADARG (index out of range, negative or non-finite rate, n < 0, bad mode), NOMEM
 * (pinned staging), CUDA. */
int aton_add_sources(aton_handle h, const int64_t* cell_idx, const double* rate_per_s,
                     int64_t n, int mode);

/* Queues nsteps radiative steps on the handle's stream (asynchronous). Each step is the
 * transport of (N, F) from the old state, the clamp N >= 0, |F| <= cN, source injection and
 * the chemistry/cooling/absorption operator per cell. Errors: BADARG (nsteps < 0), STATE
 * (fields not set), CUDA (launch failure), or a SUBCYCLE/NONFINITE status latched by an
 * earlier synchronising call. */
int aton_step(aton_handle h, int nsteps);

/* Waits for queued work and returns its status: ATON_ERR_SUBCYCLE or ATON_ERR_NONFINITE if a
 * cell was flagged since the last aton_set_fields, else OK or a CUDA error. */
int aton_synchronize(aton_handle h);

/* Returns the photon budget [photons], indices ATON_B_*; out must hold ATON_BUDGET_LEN
 * doubles. Reductions are FP64 and in a fixed order (deterministic). Synchronises. */
int aton_photon_budget(aton_handle h, double* out);

/* The photon budget without stalling the stream: aton_budget_request queues the reductions of
 * the budget as of the work queued so far, and a device-to-host copy into the handle's pinned
 * buffer, and returns at once; aton_budget_collect waits for that copy (only) and returns the
 * same vector aton_photon_budget would have returned at the request. A driver that requests
 * after each step and collects the previous request keeps the GPU busy while it reads the
 * budget of every step. One request is outstanding at a time (a new request replaces one not
 * collected); collect without a request is STATE.
 * Errors: STATE (no fields; collect without a request), CUDA (including a pipeline wait that
 * gave up, reported at collect). */
int aton_budget_request(aton_handle h);
int aton_budget_collect(aton_handle h, double* out);

/* Restores a budget saved by aton_photon_budget (checkpoint/restart); the STORED entry is
 * ignored (it is recomputed from the fields). */
int aton_set_budget(aton_handle h, const double* in);

/* Counters since aton_set_fields (synchronises). */
int aton_get_diag(aton_handle h, aton_diag* out);

/* Number of cell-steps flagged SUBCYCLE or NONFINITE since aton_set_fields (synchronises). */
int aton_last_error_cells(aton_handle h, int64_t* count);

/* Number of kernel launches per radiative step of the current execution mode. */
int aton_launches_per_step(aton_handle h, int* launches);

/* Photon count sum(N) * cell_volume [photons] of a float32 device field N of n cells, summed
 * in FP64 in a fixed order, written to *out (host memory). The paper has no counterpart: this
 * entry point exists for callers that cannot let a library allocate device memory (a host
 * code that hands out all device memory from its own fixed pool, or a hook run between time
 * steps where an allocation could block on queued work). It calls no cudaMalloc, cudaFree or
 * other allocating routine: its scratch is a fixed file-scope device array of 16384 FP64
 * partial sums plus a result slot (about 128 KB), held by every GPU that loads the library
 * until the process exits, so n is limited to 16384 * 65536 = 2^30 cells (1024^3).
 * N must be device memory of the current device; `stream` is a cudaStream_t (NULL: the
 * legacy default stream); the call enqueues two kernels and a copy on it and waits for them.
 * The first call on each device looks up the scratch address (cudaGetSymbolAddress with that
 * device current); make that first call before any stream capture. All calls share the one
 * scratch array (each call rewrites every slot it reads), so calls that overlap on the GPU
 * (from several host threads or streams at once) race and give wrong sums.
 * Errors: BADARG (NULL pointer, n < 1 or n > 2^30, cell_volume not positive and finite, N not
 * device memory of the current device), CUDA. */
int aton_photon_sum_static(const float* N, int64_t n, double cell_volume, double* out,
                           void* stream);

/* ---- chemistry surrogate (a learned replacement of the chemistry sub-cycle; not in the paper) ----
 * A 5 -> 64 -> 64 -> 3 SiLU network on BF16 tensor cores (FP32 accumulation) that replaces the
 * sub-cycled chemistry operator Phi (Appendix Eq. A4) for cells that would sub-cycle heavily.
 * Features: (log10 nH, log10 y, log10 T, log10 N, log10 dt); targets: the changes of log10 y,
 * log10 T and log10 N over dt; both standardised by aton_mlp_fit_norm. Parameters are one
 * float vector (W1 64x5, b1, W2 64x64, b2, W3 3x64, b3; aton_mlp_num_params() floats). Pair
 * records are 8 floats: nH, N, y, T (operator input), N', y', T' (output), sub-steps taken.
 * All array arguments are device pointers unless `where` says otherwise; calls synchronise. */

/* Records, for every `stride`-th cell (offset rotating with the step), the chemistry operator's
 * input and output at each following step into `records` (device, capacity records of 8
 * floats; NULL stops). Step s writes slots [s P, (s+1) P), P = ceil(ncell / stride), record
 * j of cell j * stride + (s mod stride); slots whose cell falls beyond the grid are left as
 * they were. While set, steps run the plain three-kernel path without graphs. */
int aton_set_pair_sink(aton_handle h, float* records, int64_t capacity, int stride);
int aton_pair_count(aton_handle h, int64_t* count);

/* Uses network m in the chemistry of later steps (NULL or enabled = 0: off). The handle keeps
 * the pointer; m must outlive its use. In ATON_MODE_FUSED with the GLF flux and nx a multiple
 * of 4 the step stays one launch: the TMA-staged fused kernel lists the cells its gate selects
 * (cells off the one-sub-step chemistry shortcut only) and runs the network for them at the end
 * of each CTA; otherwise (ATON_MODE_UNFUSED, ATON_MODE_FUSED_LDG, the HLL flux, nx not a
 * multiple of 4) the step runs the plain path with a gate pass and a surrogate pass
 * (aton_launches_per_step reports which). A cell is offered to the network when its explicit
 * sub-step estimate from photo-ionisation and photo-heating is >= gate_substeps and its features
 * lie in the training range; a prediction is accepted when its photons absorbed per atom match
 * the atoms ionised plus the recombinations over dt within residual_max of max(y, 1e-8); every
 * other cell takes the exact operator. The first fused step after this call (or after a change
 * of tile) allocates the per-tile lists (64 cells of 32 bytes per tile). */
void aton_default_surrogate_params(aton_surrogate_params* p);
int aton_set_surrogate(aton_handle h, aton_mlp_handle m, const aton_surrogate_params* p);

int aton_mlp_create(aton_mlp_handle* out, unsigned long long seed);
void aton_mlp_destroy(aton_mlp_handle m);
int aton_mlp_num_params(void);
int aton_mlp_set_params(aton_mlp_handle m, const float* theta, int where);
int aton_mlp_get_params(aton_mlp_handle m, float* theta, int where);
/* standardisation from pair records; the normalisation block is 26 floats: input mean[5],
 * scale[5], output mean[3], scale[3], input min[5], max[5] */
int aton_mlp_fit_norm(aton_mlp_handle m, const float* records, int64_t n, double dt);
int aton_mlp_get_norm(aton_mlp_handle m, float* out);
int aton_mlp_set_norm(aton_mlp_handle m, const float* in);
/* standardised features X (n x 5) and targets T (n x 3, may be NULL) of pair records */
int aton_mlp_features(aton_mlp_handle m, const float* records, int64_t n, double dt, float* X,
                      float* T);
/* network outputs Y (n x 3) of standardised features X */
int aton_mlp_forward(aton_mlp_handle m, const float* X, int64_t n, float* Y);
/* mean squared error and its gradient (device, num_params floats) over a batch */
int aton_mlp_loss_grad(aton_mlp_handle m, const float* X, const float* T, int n, float* grad,
                       double* loss);
/* one Adam step (beta 0.9, 0.999, eps 1e-8) on a batch; loss may be NULL (no wait) */
int aton_mlp_train_step(aton_mlp_handle m, const float* X, const float* T, int n, float lr,
                        double* loss);
int aton_mlp_synchronize(aton_mlp_handle m);

/* ---------------------------------------------------------------------------------------
 * Ionisation and radiation statistics of the current state (section 4: the volume-weighted
 * ionised fraction x_v and the distribution of the neutral fraction; the mean intensity J21
 * and the photo-ionisation rate Gamma12 and their distribution; the density dependence
 * (1-x)(nH) and J21(nH) with the mean per density bin, compared with photo-ionisation
 * equilibrium under a uniform or self-shielded field).
 *
 * Readings: Gamma = c sigma_n N (no sub-grid clumping factor), Gamma12 = Gamma / 1e-12 s^-1.
 * J21 is the Lyman-limit mean intensity, in 1e-21 erg s^-1 cm^-2 Hz^-1 sr^-1, of a spectrum
 * J_nu = J_0 (nu/nu_0)^-alpha with the same photo-ionisation rate when sigma falls as nu^-3:
 * Gamma = 4 pi J_0 sigma_0 / (h (alpha + 3)), sigma_0 = 6.30e-18 cm^2.
 * Histograms use log-spaced bins: edge k of a quantity with range [lo, hi] and nb bins is
 * 10^(log10 lo + k (log10 hi - log10 lo) / nb) rounded to float; a value v lies in bin b when
 * edge[b] <= v < edge[b+1], values below edge[1] count in bin 0 and values at or above
 * edge[nb-1] in bin nb-1. The decision compares the stored float values with the float edges
 * (J21 bins compare N with the edges divided by the J21-per-N factor), so it is exact.
 * --------------------------------------------------------------------------------------- */
#define ATON_STATS_MAX_BINS 64

typedef struct {
  int nb_nH, nb_y, nb_J;      /* bins of nH, of the neutral fraction y = 1-x, of J21 (1..64) */
  double nH_lo, nH_hi;        /* [cm^-3] range of the density bins */
  double y_lo, y_hi;          /* range of the neutral-fraction bins */
  double J21_lo, J21_hi;      /* range of the J21 bins */
  double spectral_index;      /* alpha of the J21 reading (default 1) */
  double nH_plateau;          /* J21 plateau J0: mean over cells with nH below this (1e-3) */
} aton_stats_params;

typedef struct {
  double x_volume, x_mass;        /* volume-weighted and mass-weighted ionised fraction */
  double gamma12_volume;          /* volume-averaged Gamma12 */
  double J21_volume, J21_plateau; /* volume-averaged J21; its mean over nH < nH_plateau */
  double T_volume, T_mass;        /* volume- and mass-weighted temperature [K] */
  double photons;                 /* sum N V */
  int64_t cells, plateau_cells;
} aton_stats;

/* Defaults: 48 density bins over [1e-6, 1] cm^-3, 48 neutral-fraction bins over [1e-7, 1],
 * 48 J21 bins over [1e-6, 1e4], alpha = 1, plateau below 1e-3 cm^-3. */
int aton_default_stats_params(aton_stats_params* p);

/* Statistics of the state after the steps queued so far (waits for them). Host output arrays,
 * each may be NULL: hist_y [nb_nH][nb_y] and hist_J [nb_nH][nb_J] cell counts (row-major,
 * density bin first), bin_count [nb_nH] cells per density bin, bin_mean_y and bin_mean_J21
 * [nb_nH] volume averages of y and J21 per density bin (0 where the bin is empty).
 * One pass over N, y, T, nH (16 bytes per cell) in device kernels; counts and histograms are
 * exact, sums are per-thread compensated FP32 reduced in FP64 in a fixed order (deterministic).
 * Errors: BADARG (NULL handle, params or stats; bins outside 1..64; a range with lo <= 0 or
 * hi <= lo), STATE (no fields), NOMEM, CUDA. */
int aton_ionisation_stats(aton_handle h, const aton_stats_params* p, aton_stats* s,
                          uint64_t* hist_y, uint64_t* hist_J, uint64_t* bin_count,
                          double* bin_mean_y, double* bin_mean_J21);

/* Neutral fraction in photo-ionisation equilibrium, (1-x) Gamma(nH) = alpha_B(T) nH x^2
 * (section 3.2.1, Eq. 14 at steady state, no collisional ionisation), for the field models of
 * section 4: Gamma(nH) = Gamma_0 exp(-(nH/n_star)^power), power 0 (uniform J0), 1 (J1) or 4
 * (J4; read as exp(-(nH/n*)^4), the form of the figure caption), with Gamma_0 the rate of
 * J21_0 under the reading above and alpha_B the Hui & Gnedin (1997) case-B fit. Written without
 * cancellation: x = 2G / (G + sqrt(G^2 + 4 a G)), y = a x^2 / G with G = Gamma, a = alpha nH.
 * Host computation (a closed form per density value). Errors: BADARG (NULL arrays, n < 0,
 * J21_0 < 0, T <= 0, n_star <= 0 with power > 0, power not 0, 1 or 4, alpha <= -3). */
int aton_equilibrium_neutral_fraction(const double* nH, int n, double J21_0, double n_star,
                                      int power, double T, double spectral_index,
                                      double* y_out);

/* ---------------------------------------------------------------------------------------
 * Source model of the post-processing (section 2.3): star particles of snapshot p+1 emit over
 * the interval [t_p, t_{p+1}] (length D) at a rate that spreads the photons they emit inside it
 * over the whole interval. A star of lifetime L emits Q = photons_per_baryon * mass / m_H
 * photons uniformly over its lifetime, Ndot = Q / L. With a = its age at t_{p+1} and
 * a_p = a - D its age at t_p:
 *   a_p >= L       no emission (cell -1, rate 0);
 *   a_p < 0        born inside the interval, emits for min(a, L): rate = min(a, L)/D Ndot;
 *   0 <= a_p < L   emits for min(D, L - a_p): rate = min(D, L - a_p)/D Ndot.
 * Readings: the printed "(a_{p+1} - a*)" and "min(1, L - a_p)" mix an age with a time and a
 * number with a time; the emitting time inside the interval is read instead, which keeps
 * every star's photons exact. The effective rate is Ndot_eff = rate f_esc B(t) (Eq. 16) with
 * the boost factor B(t) = max(1, a_b exp(k_b / t)) (Eq. 17 prints min, which would make the
 * boost never exceed 1; its table's a_b and k_b only boost with max), t the age of the Universe.
 * The cell is the nearest grid point, floor(x/dx) wrapped periodically.
 * --------------------------------------------------------------------------------------- */
typedef struct {
  double x, y, z;             /* position [cm] */
  double mass;                /* stellar mass [g] */
  double age;                 /* age at the end of the interval, a_{p+1} [s] (>= 0) */
  double lifetime;            /* ionising lifetime L [s] (> 0; drawn by the caller) */
  double photons_per_baryon;  /* ionising photons per stellar baryon over the lifetime */
} aton_star;

typedef struct {
  double interval;            /* D = t_{p+1} - t_p [s] (> 0) */
  double f_esc;               /* escape fraction (>= 0) */
  double boost_a, boost_k;    /* B = max(1, boost_a exp(boost_k / t)); boost_a <= 0: B = 1 */
  double t_universe;          /* age of the Universe [s] at which B is evaluated (> 0) */
} aton_source_model;

/* Cell (-1 when the star is not active inside the interval: zero emitting time) and effective
 * rate [photons/s] of each star, for a grid of nx*ny*nz cells of size dx. Host arrays; no
 * handle needed. The output feeds aton_add_sources (cells >= 0), which merges stars that
 * share a cell.
 * Errors: BADARG (NULL arrays with n > 0, n < 0, bad grid or model, a star with negative or
 * non-finite mass/age/photon yield, non-positive lifetime, non-finite position). */
int aton_star_sources(const aton_star* stars, int64_t n, const aton_source_model* m, int nx,
                      int ny, int nz, double dx, int64_t* cell, double* rate);

/* Static description of a status code. */
const char* aton_strerror(int code);

/* Detail of the last failure on the calling thread ("" if none). */
const char* aton_last_message(void);

#ifdef __cplusplus
}
#endif
#endif
