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
  int32_t n_cells; /* N >= 2; nodes 0..N */
  int32_t pad0;
} cp_gap;

/* External circuit (Sec. 2.1, App. A): a series R-L loop with the source
   V_s(t) = V0 (1 - cos 2 pi f t) exp(-t/tau) / 2 driving the x = 0 electrode
   with sign `polarity`; C is the load capacitance used by the weak scheme's
   free circuit solve (Sec. 2.4.3) and to derive A when area == 0. */
typedef struct {
  double R, L, C;
  double V0, f, tau;
  double polarity;
  int32_t kind; /* CP_CIRCUIT_* */
  int32_t pad0;
} cp_circuit;

/* Ion-induced SEE (Sec. 2.3) and the ion beam entering at x = d.
   Mean yield gamma(E) = min(scale * gamma_coef * sqrt(E / E_ref), gamma_max),
   count = floor(gamma) + Bernoulli(gamma - floor(gamma)), speed of each
   emitted electron = sqrt(e T_emit / m_e) |N(0,1)|, normal emission.  Beam:
   beam_per_step ions per step, energy beam_E_eV (mode 0) or uniform in
   [beam_Emin_eV, beam_Emax_eV] (mode 1).  0 <= gamma_max <= 14. */
typedef struct {
  double gamma_coef, gamma_max, E_ref_eV, scale, T_emit_eV;
  double beam_E_eV, beam_Emin_eV, beam_Emax_eV;
  int32_t beam_per_step;
  int32_t beam_mode;
} cp_see_beam;

/* Run controls.  Capacities are per species in macroparticles (0 picks a
   default from the loaded counts and max_steps). */
typedef struct {
  double dt;           /* time step [s] */
  uint64_t seed;       /* Philox4x64-10 key word 0 for SEE and beam draws */
  int64_t capacity[3]; /* particle store capacity per species */
  int64_t max_steps;   /* history rows to keep (levels 0..max_steps) */
  int32_t precision;   /* CP_FP64 or CP_FP32 */
  int32_t compact_every; /* steps between removals of absorbed particles (0 => 64) */
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
  double pad;
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

/* Advance n_steps steps with strict (monolithic) coupling, Sec. 2.4.2: the
   circuit's Schur row Q^n = K - g phi_0^n is folded into the x = 0 Poisson row
   (Eq. Poisson_BC2) and the coupled system is solved directly, then refined
   until its backward error (Poisson rows and circuit row) is <= residual_tol
   (at most 3 refinement sweeps).  The first call also deposits the loaded
   particles and solves level 0.  Errors: CP_ERR_ARG, CP_ERR_CAPACITY,
   CP_ERR_RESIDUAL, CP_ERR_NONFINITE, CP_ERR_CUDA. */
int cp_step_strict(cp_ctx* ctx, int32_t n_steps, double residual_tol);

/* Advance n_steps steps with weak (one-step-lagged, operator-split)
   coupling, Sec. 2.4.3: the free circuit gives Q*^n (load capacitor C), which
   enters Eq. Poisson_BC3; afterwards Q^n := C phi_0^n.  Strict and weak calls
   may be interleaved.  Errors as cp_step_strict. */
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
   capacity se_cap).  counts (device, 6 int64): ions absorbed at x = 0 and
   x = d, electrons emitted at x = 0 and x = d, electrons written, and the
   convection count at x = 0.  The first call on a device looks up the
   scratch array's address; make that first call before any stream capture.
   The call synchronises `stream`.  Every call shares the one scratch array:
   calls that overlap on the GPU (other streams, other host threads) race.
   Errors: CP_ERR_ARG (null buffer, n_cells outside 2..4096, bad sizes),
   CP_ERR_CAPACITY (n > 524288 ions, the scratch's limit; or more emitted
   electrons than se_cap), CP_ERR_CUDA. */
int cp_push_ions_noalloc(const cp_gap* gap, const cp_see_beam* see, double dt, uint64_t seed,
                         int64_t step, int32_t half_kick, const double* E, float* xi, float* u,
                         const uint32_t* id, int64_t n, int64_t* G, float* se_xi, float* se_u,
                         int64_t se_cap, int64_t* counts, void* stream);

void cp_destroy(cp_ctx* ctx);
const char* cp_status_str(int status);

#ifdef __cplusplus
}
#endif

#endif /* CP_H */
