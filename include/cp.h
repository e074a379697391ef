/*
 * cp.h -- C ABI of the GB300 (sm_103a) circuit-coupled electrostatic PIC
 * step with ion-induced secondary electron emission (SEE).
 *
 * What one step computes (arXiv 2603.24010):
 *   gather of the half-grid field at each particle (App. C), leapfrog push
 *   (Sec. 2.2.2, Eqs. vel_update_main / pos_update_main), absorption at the
 *   electrodes with ion-energy-dependent SEE folded into the convection
 *   charge (Sec. 2.3, Algorithm see_sampling_1d; Sec. 2.4.1, Eq. for
 *   Q_conv^n), injection of a beam of ions at x = d, cloud-in-cell charge
 *   deposition with the boundary-node rule of App. E.2, and the Poisson solve
 *   whose x = 0 row carries the surface charge set by the external circuit
 *   (App. B; Sec. 2.4.2 Eq. Poisson_BC2 for strict coupling, Sec. 2.4.3
 *   Eq. Poisson_BC3 for weak coupling).
 *
 * Geometry and units.  The driven electrode is at x = 0 (node 0) and the
 * grounded electrode at x = d (node N, phi_N = 0).  Particles are stored in
 * cell units: xi = x/dx in (0, N) and u = v dt/dx (cells per step).  Species
 * 0 = plasma electrons, 1 = ions (charge +e, mass m_i), 2 = secondary
 * electrons.  Every macroparticle carries the same weight.  Charge is
 * deposited as int64 fixed point (2^16 per macroparticle, positions resolved
 * to 2^-16 of a cell inside the deposit), so the charge grid is bit-identical
 * from run to run and independent of particle order.
 *
 * Memory and streams.  The library owns all device memory it allocates in
 * cp_create; the caller owns every host buffer passed in, which is only read
 * or written during the call.  Work is issued on the caller's CUDA stream
 * (cudaStream_t passed as void*, NULL = legacy default stream).  Every
 * function returns CP_OK (0) or a negative CP_ERR_* code; cp_status_str()
 * names it.  Step calls synchronise the stream before returning so that the
 * device-side status (capacity overflow, residual, non-finite field) is
 * reported by the call that met it; after such an error the context stops
 * advancing and stays at the last level it reached.
 *
 * Threading: a context must not be used from two host threads at once.
 */
#ifndef CP_H
#define CP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CP_OK 0
#define CP_ERR_ARG (-1)       /* invalid argument or call order */
#define CP_ERR_OOM (-2)       /* device allocation failed */
#define CP_ERR_CUDA (-3)      /* a CUDA runtime call failed */
#define CP_ERR_CAPACITY (-4)  /* a particle store or scratch list overflowed */
#define CP_ERR_RESIDUAL (-5)  /* strict solve missed the requested residual */
#define CP_ERR_NONFINITE (-6) /* NaN/Inf in the field or circuit state */
#define CP_ERR_TIMEOUT (-7)   /* reserved: a bounded device wait gave up */

#define CP_ELECTRONS 0
#define CP_IONS 1
#define CP_SECONDARIES 2

#define CP_FP64 0 /* particles and gather/push in FP64 */
#define CP_FP32 1 /* particles and gather/push in FP32; field/circuit in FP64 */

#define CP_CIRCUIT_SERIES_RLC 0 /* L Q'' + R Q' + V_gap = polarity V_s(t) */
#define CP_CIRCUIT_OPEN 1       /* floating driven electrode: Q_circ constant */
#define CP_CIRCUIT_TESLA 2      /* the paper's 5-loop Tesla transformer (cp_tesla) */

#define CP_UNITS_CELL 0 /* xi = x/dx, u = v dt/dx */
#define CP_UNITS_SI 1   /* x [m], v [m/s] */

/* Gap, electrodes and particle species (Sec. 2.2, App. B, Table 2). */
typedef struct {
  double d;      /* electrode separation [m] */
  double area;   /* electrode area A [m^2]; 0 => C d / eps0 (gap is the capacitor C) */
  double eps0;   /* [F/m] */
  double e;      /* elementary charge [C] */
  double m_e;    /* electron mass [kg] */
  double m_i;    /* ion mass [kg], singly charged */
  double weight; /* physical particles per macroparticle (all species) */
  double sigma0; /* surface charge density on x = 0 before the first step [C/m^2] */
  int32_t n_cells; /* N >= 2; nodes 0..N.  At most what the push's shared
                      memory holds: 11,390 cells with FP32 particles and
                      7,231 with FP64 on a GB300 (227 KB per CTA); larger
                      gaps are refused with CP_ERR_ARG */
  int32_t pad0;
} cp_gap;

/* The simplified Tesla transformer of Sec. 2.1 (Eqs. loop_1-loop_5, the
   parameters of Table 3): loop charges Q1..Q5 with
     Q1/C1 + R1 (Q1 - Q2 - Q5)' = 0
     R1 (-Q1 + Q2 + Q5)' + R2 Q2' + L1 Q2'' + M Q3'' = 0
     M Q2'' + L2 Q3'' + R3 (Q3 - Q4 + Q5)' = 0
     R3 (-Q3 + Q4 - Q5)' + V_C3 = 0           (V_C3 = Q4/C3 alone; phi_0 coupled)
     R1 (-Q1 + Q2 + Q5)' + Q5/C2 + R3 (Q3 - Q4 + Q5)' = 0
   discretised by BDF2 (App. A; the matrix and history terms are formed from
   these equations).  The gap is the load capacitor C3, its electrode charge
   Q_circ = Q4 (Sec. 2.4.2); strict coupling folds Q4 = K - [T'^{-1}]_44 phi_0
   into the x = 0 row (Eqs. Q4_phi_relation, K_def, Poisson_BC2), weak
   coupling advances the loops alone with C3's voltage starting from phi_0 of
   the previous level.  Before t = 0 the circuit rests with only C1 charged,
   to V1; the first step redistributes that charge around the capacitor loop
   C1-C2-C3.  All values SI and > 0 except M >= 0 (M^2 < L1 L2). */
typedef struct {
  double R1, R2, R3;
  double C1, C2, C3;
  double L1, L2, M;
  double V1; /* initial voltage of C1 [V] */
} cp_tesla;

/* External circuit (Sec. 2.1, App. A).  kind CP_CIRCUIT_SERIES_RLC: a series
   R-L loop with the source V_s(t) = V0 (1 - cos 2 pi f t) exp(-t/tau) / 2
   driving the x = 0 electrode with sign `polarity`; C is the load
   capacitance used by the weak scheme's free circuit solve (Sec. 2.4.3) and
   to derive A when area == 0.  kind CP_CIRCUIT_TESLA: `tesla` (R, L, C, V0,
   f, tau and polarity unused; the load capacitance is tesla.C3). */
typedef struct {
  double R, L, C;
  double V0, f, tau;
  double polarity;
  int32_t kind; /* CP_CIRCUIT_* */
  int32_t pad0;
  cp_tesla tesla;
} cp_circuit;

/* Ion-induced SEE (Sec. 2.3, Algorithm see_sampling_1d) and the ion beam
   entering at x = d.  Mean yield gamma(E) = min(scale * gamma_coef *
   sqrt(E / E_ref), gamma_max) (the paper's fitted polynomial has no
   published coefficients; this law stands in), 0 <= gamma_max <= 14.
   Count: count_law CP_SEE_COUNT_BERNOULLI floor(gamma) + Bernoulli(gamma -
   floor(gamma)), or CP_SEE_COUNT_POISSON Poisson(gamma) as in the paper,
   sampled by inversion of its distribution function (at most 64 electrons).
   Speed of each emitted electron: energy_law CP_SEE_ENERGY_MAXWELL
   sqrt(e T_emit / m_e) |N(0,1)|, or CP_SEE_ENERGY_LOGNORMAL as in the paper:
   energy E = exp(ln_mu + ln_sigma N(0,1)) eV, speed sqrt(2 E e / m_e) (the
   paper's fitted mu, sigma are not published).  Normal emission.  Beam:
   beam_per_step ions per step, energy beam_E_eV (mode 0) or uniform in
   [beam_Emin_eV, beam_Emax_eV] (mode 1). */
typedef struct {
  double gamma_coef, gamma_max, E_ref_eV, scale, T_emit_eV;
  double beam_E_eV, beam_Emin_eV, beam_Emax_eV;
  int32_t beam_per_step;
  int32_t beam_mode;
  int32_t count_law;  /* CP_SEE_COUNT_* */
  int32_t energy_law; /* CP_SEE_ENERGY_* */
  double ln_mu, ln_sigma; /* lognormal law: ln(E / 1 eV) ~ N(ln_mu, ln_sigma^2) */
} cp_see_beam;

#define CP_SEE_COUNT_BERNOULLI 0
#define CP_SEE_COUNT_POISSON 1
#define CP_SEE_ENERGY_MAXWELL 0
#define CP_SEE_ENERGY_LOGNORMAL 1

/* Run controls.  Capacities are per species in macroparticles (0 picks a
   default from the loaded counts and max_steps). */
typedef struct {
  double dt;           /* time step [s] */
  uint64_t seed;       /* Philox4x64-10 key word 0 for SEE and beam draws */
  int64_t capacity[3]; /* particle store capacity per species */
  int64_t max_steps;   /* history rows to keep (levels 0..max_steps) */
  int32_t precision;   /* CP_FP64 or CP_FP32 */
  int32_t compact_every; /* steps between removals of absorbed particles (0 => 128) */
} cp_run;

/* One diagnostics row per time level n (written by the solve at t_n). */
typedef struct {
  int64_t step;
  double t;
  double V_gap;      /* phi_0^n [V] */
  double I_circ;     /* circuit current: BDF2 derivative of the circuit charge [A] */
  double Q_surf;     /* sigma_+^n A [C] */
  double Q_conv;     /* convection charge into x = 0 over (t_{n-1}, t_n] [C] */
  double Q_circ;     /* Q_circ^n [C] */
  double V_source;   /* polarity V_s(t_n) [V] */
  double residual;   /* backward error of the coupled solve */
  double ion_energy_eV; /* energy of the ions absorbed at x = 0 in the push */
  double max_cfl;    /* max |u| (cells/step) in the push that produced level n */
  double J_hat;      /* learned weak scheme: predicted plasma charge used at this
                        level (0 when the plain lagged solve was used) [C] */
  int64_t absorbed[2][3]; /* [x = 0, x = d][species] */
  int64_t emitted[2];     /* secondaries emitted at [x = 0, x = d] */
  int64_t injected;       /* beam ions appended */
  int64_t n_live[3];      /* live macroparticles per species at level n */
  int64_t conv_count;     /* Q_conv / (e weight) */
} cp_diag;

typedef struct cp_ctx cp_ctx;

/* Create a gap instance on the current CUDA device.  Allocates the particle
   stores, grids and history on the device.  `stream` is a cudaStream_t (may
   be NULL).  On success *out owns the context (free with cp_destroy).
   Errors: CP_ERR_ARG (N < 2, d/dt/weight <= 0, unknown enum), CP_ERR_OOM. */
int cp_create(const cp_gap* gap, const cp_circuit* circuit, const cp_see_beam* see,
              const cp_run* run, void* stream, cp_ctx** out);

/* Load the macroparticles of one species before the first step (replaces any
   previous set of that species).  x, v: host arrays of n values in `units`;
   id: host array of n ion ids (ions only; NULL => 0..n-1) -- ids key the SEE
   random draws, and beam ions are numbered from max(id)+1.  Every x must lie
   strictly inside the gap.  Values are rounded to the store's precision.
   Errors: CP_ERR_ARG (bad species/units, particle outside, after the first
   step), CP_ERR_CAPACITY (n exceeds the store), CP_ERR_CUDA. */
int cp_set_particles(cp_ctx* ctx, int32_t species, const double* x, const double* v,
                     const uint32_t* id, int64_t n, int32_t units);

/* Initial plasma (the paper's runs start from a gap filled with a uniform
   plasma, Sec. 3.1; density and temperature are the workload's).  n_pairs
   co-located electron/ion pairs, so the initial charge density is exactly
   zero: pair k is drawn from Philox4x64-10 counter (k, 0, 0, 0) under key
   (seed, load tag 0x4C4F4144); draw 0 places it uniformly in the gap
   (xi = N u0, rounded to the store's precision, kept inside (0, N)) and the
   Box-Muller pair of draws 1 and 2, z_e = r cos(2 pi u2), z_i = r sin(2 pi
   u2) with r = sqrt(-2 ln u1), gives the velocities z sqrt(e T_load / m)
   (a Maxwellian of temperature T_load in 1D, per species).  Ion k gets id k.
   Weight: `weight` if > 0, else n0 d A / n_pairs if n0 > 0, else the gap's
   weight is kept; a new weight replaces cp_gap.weight for every species and
   the beam. */
typedef struct {
  double n0;        /* plasma density [m^-3] (0: keep the weight) */
  double T_load_eV; /* temperature of both species [eV] */
  int64_t n_pairs;  /* electron/ion pairs (0 <= n_pairs < 2^32) */
  double weight;    /* physical particles per macroparticle (0: from n0) */
} cp_species;

/* Draw the initial plasma on the device (no host particle arrays, nothing
   copied from the host).  Replaces any electrons and ions staged by
   cp_set_particles; call before the first step (the draw runs when the first
   step call allocates the stores).  Afterwards cp_set_particles accepts only
   the secondaries.  Errors: CP_ERR_ARG (after the first step, n_pairs out of
   range, negative or non-finite T_load_eV, n0 or weight), CP_ERR_CAPACITY
   (n_pairs above a requested electron or ion capacity). */
int cp_load_species(cp_ctx* ctx, const cp_species* species, uint64_t seed);

/* Advance n_steps steps with strict (monolithic) coupling, Sec. 2.4.2: the
   circuit's Schur row Q^n = K - g phi_0^n is folded into the x = 0 Poisson row
   (Eq. Poisson_BC2) and the coupled system is solved directly, then refined
   until its backward error (Poisson rows and circuit row) is <= residual_tol
   (at most 3 refinement sweeps).  The first call also deposits the loaded
   particles and solves level 0.  Errors: CP_ERR_ARG, CP_ERR_CAPACITY,
   CP_ERR_RESIDUAL, CP_ERR_NONFINITE, CP_ERR_CUDA. */
int cp_step_strict(cp_ctx* ctx, int32_t n_steps, double residual_tol);

/* Advance n_steps steps with weak (one-step-lagged, operator-split)
   coupling, Sec. 2.4.3: the circuit alone is advanced first, its load
   capacitor C starting from the electrode potential of the previous level
   (the capacitor state handed back to the circuit, Q_4^{n-1} = C phi_0^{n-1})
   while the circuit keeps its own loop-charge history:
     a21 Q^n - hist + phi_0^{n-1} + (Q^n - Q^{n-1})/C = polarity V_s(t_n),
   a21 and hist being the BDF2 terms of the strict scheme.  The capacitor
   charge Q*^n = C phi_0^{n-1} + Q^n - Q^{n-1} then enters Eq. Poisson_BC3
   (the circuit delivers Q^n - Q^{n-1} to the electrode).  Without plasma
   this equals the strict solve; with plasma it lags the strict one by the
   plasma's own change of C phi_0 over the step.  Q_circ in the diagnostics
   is the loop charge Q^n in both schemes.  Strict and weak calls may be
   interleaved.  Errors as cp_step_strict. */
int cp_step_weak(cp_ctx* ctx, int32_t n_steps);

/* Current level's diagnostics row (synchronises the stream). */
int cp_read_scalars(cp_ctx* ctx, cp_diag* out);

/* Rows first_step .. first_step+n-1 (levels; 0 is the initial solve).
   Errors: CP_ERR_ARG if a row is not yet written or beyond max_steps. */
int cp_read_history(cp_ctx* ctx, int64_t first_step, int64_t n, cp_diag* out);

/* Current level's fields: phi (N+1 nodes, V), rho (N+1 nodes, C/m^3),
   E (N edges, E[k] = E_{k+1/2}, V/m) and the int64 charge grid G (N+1;
   rho = G e weight / (A dx 2^16)).  Any pointer may be NULL.  n_nodes must be
   N+1.  Synchronises the stream. */
int cp_read_grid(cp_ctx* ctx, double* phi, double* rho, double* E, int64_t* G,
                 int32_t n_nodes);

/* Copy the live particles of one species to host arrays of capacity `cap`
   (cell units; id only for ions, may be NULL); *n receives the count.
   Order is unspecified.  Errors: CP_ERR_CAPACITY if cap is too small. */
int cp_get_particles(cp_ctx* ctx, int32_t species, double* xi, double* u, uint32_t* id,
                     int64_t cap, int64_t* n);

/* Current time level (number of completed steps). */
int cp_get_level(cp_ctx* ctx, int64_t* level);

/* Serialise the whole state (particles, circuit history, surface charge,
   level, history rows) into a host buffer.  With buf == NULL, *len receives
   the size needed.  A state loaded into a context created with the same
   parameters continues bit-identically (counter-based random draws). */
int cp_save_state(cp_ctx* ctx, void* buf, size_t* len);
int cp_load_state(cp_ctx* ctx, const void* buf, size_t len);

/* Number of kernels the last step call launched (for accounting of
   launches in benchmarks). */
int cp_last_launch_count(cp_ctx* ctx, int64_t* launches);

/* Per-launch timing.  While on != 0, step calls launch each kernel directly
   (no graph replay) bracketed by CUDA events on the context's stream, and
   accumulate the device time of each kernel kind.  cp_read_timing returns
   the totals since timing was last enabled: ms[k], n[k] = milliseconds and
   launches of the particle push (k = 0), the coupled solve (k = 1) and the
   removal of absorbed particles (k = 2). */
int cp_enable_timing(cp_ctx* ctx, int32_t on);
int cp_read_timing(cp_ctx* ctx, double ms[3], int64_t n[3]);

/* Device time of each particle-push launch of the last step call made with
   timing on, in launch order (ms[k] for the push from level L+k, L = level
   at the start of that call).  *n receives the count; at most cap values
   are written.  Errors: CP_ERR_CAPACITY if cap < count. */
int cp_read_launch_times(cp_ctx* ctx, double* ms, int64_t cap, int64_t* n);

/* Allocation-free push of one FP32 ion population through one step (the
   paper has no counterpart; this serves callers that cannot call cudaMalloc,
   e.g. a step inside a real-time loop or a process that must not grow
   device memory after start-up).  It needs no context: every input and
   output is a caller-owned device buffer, and the scratch it needs (the
   list of ions absorbed in the push) is a static device array of 8 MiB that
   every GPU loading this library holds until the process exits.
   Computes what one cp_step call does for ions alone: gather of the field E
   (N FP64 edge values E_{k+1/2}, device), kick (half kick if half_kick != 0)
   and drift of xi/u (device, FP32 cell units, updated in place; absorbed
   ions become xi = -1), secondary emission with the Philox draws of
   (seed, step, id[k]), and the deposit of the surviving ions and the
   emitted electrons into G (device, N+1 int64, overwritten; 2^16 per
   macroparticle).  Emitted electrons are written to se_xi/se_u (device,
   capacity se_cap).  counts (device, 6 int64, written on the device): ions
   absorbed at x = 0 and x = d, electrons emitted at x = 0 and x = d,
   electrons written (at most se_cap), and the convection count at x = 0.  The first call on a device looks up the
   scratch array's address; make that first call before any stream capture.
   The call synchronises `stream`.  Every call shares the one scratch array:
   calls that overlap on the GPU (other streams, other host threads) race.
   Errors: CP_ERR_ARG (null buffer, n_cells outside 2..4096, bad sizes, a
   SEE law cp_create would refuse: gamma_max outside 0..14, a negative or
   non-finite scale, gamma_coef, E_ref_eV or T_emit_eV; a count or energy
   law other than floor + Bernoulli and the half-Maxwellian),
   CP_ERR_CAPACITY (n > 524288 ions, the scratch's limit; or more emitted
   electrons than se_cap), CP_ERR_CUDA. */
int cp_push_ions_noalloc(const cp_gap* gap, const cp_see_beam* see, double dt, uint64_t seed,
                         int64_t step, int32_t half_kick, const double* E, float* xi, float* u,
                         const uint32_t* id, int64_t n, int64_t* G, float* se_xi, float* se_u,
                         int64_t se_cap, int64_t* counts, void* stream);

/* ------------------------------------------------------------------------
 * Learned weak-coupling predictor.  The paper's weak scheme (Sec. 2.4.3)
 * lags the strict one because its circuit solve sees the capacitor voltage
 * phi_0^{n-1} + (Q^n - Q^{n-1})/C instead of phi_0^n; the difference is
 * J^n/C with J^n = C (phi_0^n - phi_0^{n-1}) - (Q^n - Q^{n-1}), the
 * plasma's own change of C phi_0 over the step (convection charge plus the
 * change of the charge the space charge induces on the electrode).  A small
 * MLP predicts J^n from the last 8 levels; the learned weak solve adds the
 * prediction J_hat to its capacitor term,
 *   a21 Q^n - hist + phi_0^{n-1} + (Q^n - Q^{n-1} + J_hat)/C = V_s,
 * which is the strict solve when J_hat = J^n.
 *
 * Network: 40 -> 64 -> 64 -> 64 -> 2, GELU (erf form) after the three
 * hidden layers, BF16 weights (rounded to nearest even from an FP32 master
 * copy), FP32 biases, FP32 accumulation.  Parameters are one FP32 array of
 * CP_MLP_NPARAM values: W1[64][40] b1[64] W2[64][64] b2[64] W3[64][64]
 * b3[64] W4[2][64] b4[2] (W[out][in], row-major).
 *
 * Features of level k (raw, one row of 5): Q_conv^k [C], phi_0^k -
 * phi_0^{k-1} [V], Q_surf^k - Q_surf^{k-1} [C], secondaries emitted at
 * x = 0 in step k, energy of the ions absorbed at x = 0 in step k [eV].  The
 * input predicting level n+1 is the rows of levels n-7..n (oldest first),
 * each value divided by in_scale of its feature.  Outputs (y0, y1) are
 * Q_conv^{n+1} / out_scale[0] (the next step's plasma current times dt) and
 * J^{n+1} / out_scale[1] (the plasma-driven increment of the electrode's
 * charge); J_hat = out_scale[1] y1, y0 being an auxiliary output.
 *
 * Fallback: the network is evaluated at every level once 8 levels of
 * features exist (in every scheme), and its error against the realised J^n
 * is tracked as exponential averages (weight 1/16) of |J^n - J_hat^n| and
 * |J^n|.  The learned solve uses J_hat only after 16 such evaluations and
 * while avg|J - J_hat| <= bound * avg|J| (bound > 0); otherwise it falls
 * back to the plain lagged solve (J_hat = 0) for that level.
 * ------------------------------------------------------------------------ */
#define CP_MLP_IN 40
#define CP_MLP_HIDDEN 64
#define CP_MLP_OUT 2
#define CP_MLP_NPARAM 11074
#define CP_PRED_WINDOW 8
#define CP_PRED_FEATURES 5

typedef struct {
  float in_scale[5];  /* divisors of the five features (> 0) */
  float out_scale[2]; /* multipliers of the two outputs (> 0) */
  float pad0;
  double bound;       /* fallback bound on avg|J - J_hat| / avg|J| (> 0) */
} cp_predictor;

/* Install a trained network in the context (params: host, CP_MLP_NPARAM
   FP32 values; rounded to BF16 on the device).  From the next solve on, the
   network is evaluated at every level and its error tracked; only
   cp_step_weak_learned uses its predictions.  Errors: CP_ERR_ARG (null
   pointers, scales <= 0 or not finite, bound <= 0), CP_ERR_CUDA. */
int cp_set_predictor(cp_ctx* ctx, const float* params, const cp_predictor* norm);

/* Advance n_steps steps with the learned weak scheme described above.
   Errors: CP_ERR_ARG if no predictor is installed; otherwise as
   cp_step_weak. */
int cp_step_weak_learned(cp_ctx* ctx, int32_t n_steps);

/* Training samples from the context's history rows: for k = 0..n-1 the
   window ending at level L = first_level + k (raw features, not divided by
   the scales) goes to X[k][0..39] and the targets of level L+1 to Y[k][0]
   = Q_conv^{L+1}, Y[k][1] = J^{L+1} [C].  X (n x 40) and Y
   (n x 2) are FP32 device arrays; values are formed in FP64 and rounded
   once.  Requires first_level >= 8 and first_level + n <= the current level.
   Stream-ordered on the context's stream.  Errors: CP_ERR_ARG. */
int cp_predictor_samples(cp_ctx* ctx, int64_t first_level, int64_t n, float* X, float* Y);

/* Training kernels.  All arrays are FP32 device arrays; work is issued on
   `stream` (cudaStream_t, may be NULL).  No call allocates memory. */

/* Initialise params (CP_MLP_NPARAM): weights uniform in +-sqrt(6/fan_in)
   (He), biases 0, from Philox4x64-10 draws keyed by seed. */
int cp_mlp_init(float* params, uint64_t seed, void* stream);

/* Feature and target scales of a data set (X: n x 40 raw, Y: n x 2 raw):
   in_scale[f] = root mean square of feature f over all samples and window
   positions, out_scale[o] = RMS of Y[:, o] (1 where the RMS is 0).  Fills
   the scales of *norm (bound untouched); synchronises the stream. */
int cp_mlp_scales(const float* X, const float* Y, int64_t n, cp_predictor* norm, void* stream);

/* Xn = X / in_scale, Yn = Y / out_scale (Y/Yn may be NULL). */
int cp_mlp_normalize(const float* X, const float* Y, int64_t n, const cp_predictor* norm,
                     float* Xn, float* Yn, void* stream);

/* Network outputs (normalised) for n normalised inputs: Yhat (n x 2). */
int cp_mlp_forward(const float* params, const float* Xn, int64_t n, float* Yhat, void* stream);

/* Loss and gradient of L = 1/(2n) sum_k sum_o (yhat_ko - y_ko)^2 with
   respect to params (the BF16-rounded weights are used in the forward and
   backward passes; the gradient is taken with respect to them and applied
   to the FP32 master copy).  grad: CP_MLP_NPARAM floats, *loss: one float
   (device).  work: cp_mlp_work_floats() floats of scratch (device).
   Deterministic: per-block partial sums are added in a fixed order. */
int64_t cp_mlp_work_floats(void);
int cp_mlp_loss_grad(const float* params, const float* Xn, const float* Yn, int64_t n,
                     float* grad, float* loss, float* work, void* stream);

/* One Adam step (Kingma & Ba 2015) at step number t >= 1:
   m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
   p -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps). */
int cp_mlp_adam(float* params, const float* grad, float* m, float* v, int64_t t, float lr,
                float beta1, float beta2, float eps, void* stream);

/* ------------------------------------------------------------------------
 * Ensemble of independent gap instances (uneven cells and particle counts,
 * their own circuits, SEE scales and beams) advanced together: per step one
 * persistent push launch over the particle tiles of every instance and one
 * solve launch with one CTA per instance, replayed from a CUDA graph.  An
 * instance advanced in the ensemble gives bit for bit the results it gives
 * as a context of its own (same per-particle arithmetic, integer charge,
 * counter-based draws, exact integer solve).
 * ------------------------------------------------------------------------ */
typedef struct cp_batch cp_batch;

/* Create n instances (1 <= n <= 2048) from arrays of n parameter structs.
   All runs share precision, max_steps and compact_every (0 => 64 here: the
   small instances of an ensemble lose particles fast); n_cells <= 4096.
   Errors: CP_ERR_ARG, CP_ERR_OOM, CP_ERR_CUDA, and those of cp_create. */
int cp_batch_create(int32_t n, const cp_gap* gaps, const cp_circuit* circuits,
                    const cp_see_beam* sees, const cp_run* runs, void* stream, cp_batch** out);

/* As cp_set_particles for instance i, before the first step. */
int cp_batch_set_particles(cp_batch* b, int32_t i, int32_t species, const double* x,
                           const double* v, const uint32_t* id, int64_t n, int32_t units);

/* Advance every instance n_steps steps (strict / weak coupling as in
   cp_step_strict / cp_step_weak).  An instance that meets an error stops
   (the others go on); the call returns the first non-zero instance status,
   cp_batch_status gives all of them. */
int cp_batch_step_strict(cp_batch* b, int32_t n_steps, double residual_tol);
int cp_batch_step_weak(cp_batch* b, int32_t n_steps);

/* Learned weak coupling in an ensemble (Sec. 2.4.3 with the predicted
   plasma term of cp_set_predictor): install a network on instance i (same
   arguments and errors as cp_set_predictor, any time; each instance has its
   own network and window), and advance every instance with the learned
   weak scheme.  An instance without a network runs the plain weak scheme,
   as cp_step_weak.  The ensemble's solve runs the network in the same CTA
   after the commit; results are those of the instance's own context. */
int cp_batch_set_predictor(cp_batch* b, int32_t i, const float* params, const cp_predictor* norm);
int cp_batch_step_weak_learned(cp_batch* b, int32_t n_steps);

/* Training samples of instance i, as cp_predictor_samples: an ensemble of
   strict runs generates the predictor's training set in one pass. */
int cp_batch_predictor_samples(cp_batch* b, int32_t i, int64_t first_level, int64_t n, float* X,
                               float* Y);

/* Per-instance readers, as their single-context counterparts. */
int cp_batch_read_history(cp_batch* b, int32_t i, int64_t first, int64_t n, cp_diag* out);
int cp_batch_read_grid(cp_batch* b, int32_t i, double* phi, double* rho, double* E, int64_t* G,
                       int32_t n_nodes);
int cp_batch_get_particles(cp_batch* b, int32_t i, int32_t species, double* xi, double* u,
                           uint32_t* id, int64_t cap, int64_t* n);
int cp_batch_status(cp_batch* b, int32_t* status /* n entries */);
int cp_batch_get_level(cp_batch* b, int32_t i, int64_t* level);
int cp_batch_last_launch_count(cp_batch* b, int64_t* launches);

/* Per-kernel timing of the ensemble, as cp_enable_timing / cp_read_timing:
   while on, steps launch each kernel directly between CUDA events; the
   totals are of the push (k = 0), the solve (1) and the removal (2). */
int cp_batch_enable_timing(cp_batch* b, int32_t on);
int cp_batch_read_timing(cp_batch* b, double ms[3], int64_t n[3]);

/* Launch shape of the ensemble push: threads per CTA (256, 512 or 1024) and
   CTAs per SM (0 = as many as fit).  Valid after the first step.
   Errors: CP_ERR_ARG if the shape cannot be resident. */
int cp_batch_set_launch(cp_batch* b, int32_t threads, int32_t ctas_per_sm);
int cp_batch_get_launch(cp_batch* b, int32_t* threads, int32_t* grid);

/* Autotuner: for each candidate shape (512x2, 512x1, 256x2, 256x1, 1024x1
   threads x CTAs per SM, those that fit) advance steps_per_shape ordinary
   steps of the run (mode 0 strict with residual_tol, 1 weak), time the
   push of each with CUDA events, and keep the fastest shape.  The steps
   count as steps of the run (results do not depend on the shape).  Outputs
   may be NULL.  Returns the first instance status. */
int cp_batch_autotune(cp_batch* b, int32_t steps_per_shape, int32_t mode, double residual_tol,
                      int32_t* threads, int32_t* ctas_per_sm, double* push_ms);

void cp_batch_destroy(cp_batch* b);

/* ------------------------------------------------------------------------
 * 2D planar gap: x normal to the electrodes (as in the 1D gap), y periodic
 * with n_cells_y cells over length_y.  The electrodes are equipotential
 * planes of area A (cp_gap.area, or C d / eps0); the gap's depth is
 * A / length_y.  Per step: gather of (E_x, E_y) by bilinear interpolation
 * on the staggered grid, leapfrog push in both directions (y wraps),
 * absorption and SEE at the electrodes (yield from the impact's kinetic
 * energy; emitted electrons start at the impact's y, normal to the wall),
 * beam ions entering at x = d with a Gaussian transverse profile
 * (beam_sigma, centre beam_y0), bilinear fixed-point deposit (2^16 x 2^16
 * per macroparticle, positions resolved to 2^-16 of a cell per axis, end
 * nodes in x doubled), and the solve: the transverse mean
 * is the 1D coupled problem (strict or weak, with the circuit, exactly as
 * cp_step_strict / cp_step_weak) and the other transverse Fourier modes
 * solve tridiagonal systems in x with phi = 0 on both electrodes.  The
 * particle store is kept sorted by 32 x 32-cell tiles, re-sorted every
 * sort_every steps (0 => 16).  FP32 particles only; n_cells_y a power of two
 * in 8..4096; n_cells <= 4096.
 * ------------------------------------------------------------------------ */
typedef struct {
  int32_t n_cells_y;
  int32_t sort_every;
  double length_y;   /* [m] */
  double beam_sigma; /* [m] */
  double beam_y0;    /* [m] */
} cp_transverse;

typedef struct cp_gap2d cp_gap2d;

int cp2d_create(const cp_gap* gap, const cp_transverse* tr, const cp_circuit* circuit,
                const cp_see_beam* see, const cp_run* run, void* stream, cp_gap2d** out);
/* Particles of one species before the first step: x, y, vx, vy (cell units
   xi = x/dx, eta = y/dy, u = vx dt/dx, w = vy dt/dy, or SI), ids as in
   cp_set_particles.  Errors: CP_ERR_ARG. */
int cp2d_set_particles(cp_gap2d* g, int32_t species, const double* x, const double* y,
                       const double* vx, const double* vy, const uint32_t* id, int64_t n,
                       int32_t units);
int cp2d_step_strict(cp_gap2d* g, int32_t n_steps, double residual_tol);
int cp2d_step_weak(cp_gap2d* g, int32_t n_steps);

/* Learned weak coupling of the transverse mean (the 1D coupled problem the
   2D solve contains; Sec. 2.4.3 with the predicted plasma term): install a
   network as cp_set_predictor does (its features are those of the mean:
   convection charge, V_gap and surface-charge increments, emission and
   absorbed ion energy at x = 0), and advance with the learned weak scheme.
   Errors: as cp_set_predictor / cp2d_step_weak; CP_ERR_ARG if no network
   is installed. */
int cp2d_set_predictor(cp_gap2d* g, const float* params, const cp_predictor* norm);
int cp2d_step_weak_learned(cp_gap2d* g, int32_t n_steps);
/* Diagnostics rows (V_gap = phi on the driven electrode, circuit, tallies). */
int cp2d_read_history(cp_gap2d* g, int64_t first, int64_t n, cp_diag* out);
int cp2d_get_level(cp_gap2d* g, int64_t* level);
/* Current fields, row-major over x: phi[(Nx+1) Ny], Ex[Nx Ny] at (i+1/2, j),
   Ey[(Nx+1) Ny] at (i, j+1/2), and the charge grid G[(Nx+1) Ny] of the
   level (2^32 per macroparticle).  Any pointer may be NULL.  The stores
   together hold at most 2^30 macroparticles (the int64 charge sums' range);
   cp2d_step_* refuse larger capacities with CP_ERR_ARG. */
int cp2d_read_fields(cp_gap2d* g, double* phi, float* Ex, float* Ey, int64_t* G);
/* Live particles of one species (cell units); *n receives the count.
   Errors: CP_ERR_CAPACITY if cap is too small. */
int cp2d_get_particles(cp_gap2d* g, int32_t species, double* xi, double* eta, double* u, double* w,
                       uint32_t* id, int64_t cap, int64_t* n);
/* Per-kernel-group timing while on: ms[0] push, ms[1] solve (all its
   kernels), ms[2] sort, and the number of each. */
int cp2d_enable_timing(cp_gap2d* g, int32_t on);
int cp2d_read_timing(cp_gap2d* g, double ms[3], int64_t n[3]);
int cp2d_last_launch_count(cp_gap2d* g, int64_t* launches);
void cp2d_destroy(cp_gap2d* g);

void cp_destroy(cp_ctx* ctx);
const char* cp_status_str(int status);

#ifdef __cplusplus
}
#endif

#endif /* CP_H */
