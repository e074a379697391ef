/*
 * cp_oracle.h -- plain, slow, FP64 CPU oracle of the circuit-coupled
 * electrostatic PIC step with ion-induced secondary electron emission.
 *
 * TEST INFRASTRUCTURE ONLY.  The product path never links, loads or calls
 * this code; only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline leg (and its --impl reference arm) may use it.  It shares no
 * code, header, table or constant with the CUDA path.
 *
 * Representation: particle positions are kept in cell units xi = x/dx and
 * velocities as u = v*dt/dx (cells per step).  This is a linear change of
 * variables of the paper's leapfrog (Sec. 2.2.2, Eqs. vel_update_main,
 * pos_update_main); it makes the cloud-in-cell weight of a particle exactly
 * the fractional part of xi.
 *
 * Species: 0 = plasma electrons, 1 = ions (loaded + beam), 2 = secondary
 * electrons emitted by ion impact (Sec. 2.3).
 */
#ifndef CP_ORACLE_H
#define CP_ORACLE_H

#include <stdint.h>

#define OR_SPECIES 3
#define OR_ELECTRONS 0
#define OR_IONS 1
#define OR_SECONDARIES 2

#define OR_MODE_STRICT 0
#define OR_MODE_WEAK 1
#define OR_MODE_WEAK_LEARNED 2 /* weak with the predictor's J_hat (or_set_predictor) */

#define OR_CIRCUIT_SERIES_RLC 0 /* series R-L-source into the gap */
#define OR_CIRCUIT_OPEN 1       /* floating electrode: no circuit charge */
#define OR_CIRCUIT_TESLA 2      /* the paper's 5-loop Tesla transformer (Eqs. loop_1-loop_5) */

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_RESIDUAL (-5)
#define OR_ERR_NONFINITE (-6)

/* Philox stream tags (second key word). */
#define OR_TAG_SEE 0x5345ULL
#define OR_TAG_BEAM 0x4245ULL
#define OR_TAG_LOAD 0x4C4F4144ULL

typedef struct {
  /* gap, Sec. 2.2.1 and App. B */
  double d;        /* electrode separation [m] */
  double area;     /* electrode area A [m^2] */
  double eps0;     /* vacuum permittivity [F/m] */
  double e;        /* elementary charge [C] */
  double m_e;      /* electron mass [kg] */
  double m_i;      /* ion mass [kg] (singly charged) */
  /* circuit, Sec. 2.1 and App. A (series R-L-source; see or_circuit_*) */
  double R, L, C;  /* [Ohm], [H], [F] */
  double V0, f, tau; /* source V_s(t) = V0 (1 - cos 2 pi f t) exp(-t/tau) / 2 */
  double polarity; /* sign with which V_s drives the x = 0 electrode */
  /* ion-induced SEE, Sec. 2.3 / Algorithm see_sampling_1d */
  double gamma_coef; /* gamma(E) = min(scale*coef*sqrt(E/E_ref), gamma_max) */
  double gamma_max;
  double E_ref_eV;
  double see_scale;
  double T_emit_eV;  /* temperature of the emitted half-Maxwellian [eV] */
  /* ion beam entering at x = d */
  double beam_E_eV, beam_Emin_eV, beam_Emax_eV;
  /* run */
  double dt;       /* time step [s] */
  double weight;   /* macroparticle weight (physical particles per macroparticle) */
  double sigma0;   /* initial surface charge density sigma_+^{-1} [C/m^2] */
  double grid_units; /* charge-grid units per macroparticle charge (0: 2^16, the 1D
                        deposit's; the 2D gap's transverse mean is in 2^32) */
  /* Tesla transformer (circuit == OR_CIRCUIT_TESLA, Sec. 2.1): loop charges
     Q1..Q5 of Eqs. loop_1-loop_5; the gap is the load capacitor C3 (its
     charge is Q4), C1 is pre-charged to V1 at t = 0 */
  double tR1, tR2, tR3, tC1, tC2, tC3, tL1, tL2, tM, tV1;
  /* SEE laws of Algorithm see_sampling_1d (see_count_law / see_energy_law) */
  double see_ln_mu, see_ln_sigma; /* lognormal SE energy: ln(E / 1 eV) ~ N(mu, sigma^2) */
  uint64_t seed;
  int64_t n_cells;       /* N: nodes 0..N, phi_N = 0 */
  int64_t circuit;       /* OR_CIRCUIT_* */
  int64_t beam_per_step; /* beam macroparticles appended per step */
  int64_t beam_mode;     /* 0 mono-energetic, 1 uniform in [Emin, Emax] */
  int64_t see_count_law;  /* 0 floor + Bernoulli, 1 Poisson (OR_SEE_*) */
  int64_t see_energy_law; /* 0 half-Maxwellian of T_emit, 1 lognormal */
} or_params;

#define OR_SEE_COUNT_BERNOULLI 0 /* floor(gamma) + Bernoulli(gamma - floor(gamma)) */
#define OR_SEE_COUNT_POISSON 1   /* Poisson(gamma), Algorithm see_sampling_1d */
#define OR_SEE_POISSON_MAX 64    /* truncation of the Poisson count */
#define OR_SEE_ENERGY_MAXWELL 0  /* |N(0,1)| sqrt(e T_emit / m_e) */
#define OR_SEE_ENERGY_LOGNORMAL 1 /* E = exp(mu + sigma N(0,1)) eV, v = sqrt(2 E e / m_e) */

/* Per-level diagnostics record: level n is written by the solve at t_n. */
typedef struct {
  int64_t step;
  double t;
  double V_gap;     /* phi_0^n [V] */
  double I_circ;    /* circuit current, BDF2 derivative of the circuit charge [A] */
  double Q_surf;    /* sigma_+^n * A [C] */
  double Q_conv;    /* convection charge over (t_{n-1}, t_n] [C] */
  double Q_circ;    /* Q_circ^n [C] */
  double V_source;  /* polarity * V_s(t_n) [V] */
  double residual;  /* backward error of the coupled solve */
  double ion_energy_eV; /* energy of ions absorbed at x = 0 during the push */
  double max_cfl;   /* max |u| (cells/step) over the push that produced level n */
  double J_hat;     /* learned weak scheme: prediction used at this level, else 0 [C] */
  int64_t absorbed[2][3]; /* [electrode: 0 at x=0, 1 at x=d][species] */
  int64_t emitted[2];     /* secondaries emitted at [x=0, x=d] */
  int64_t injected;       /* beam ions appended */
  int64_t n_live[3];      /* live macroparticles per species at level n */
  int64_t conv_count;     /* Q_conv / (e*w) */
} or_diag;

typedef struct or_state or_state;

/* ---- building blocks (each exported so tests can pin it) ---- */
void or_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
double or_u01(uint64_t w);
double or_source(const or_params* p, double t);
void or_deposit(int64_t N, int64_t n, const double* xi, int64_t sign, int64_t* G);
double or_gather(const double* E, int64_t N, double xi);
int or_thomas(int64_t n, const double* a, const double* b, const double* c,
              const double* r, double* x);
int64_t or_see_count(const or_params* p, double E_ion_eV, uint64_t id, int64_t step,
                     double* gamma_out);
void or_see_electron(const or_params* p, uint64_t id, int64_t step, int64_t j,
                     double* v_out, double* frac_out);
/* Loops of the two draws above over ion ids id0..id0+n-1 (test helpers). */
void or_see_count_batch(const or_params* p, double E_ion_eV, uint64_t id0, int64_t n,
                        int64_t step, int64_t* counts);
void or_see_electron_batch(const or_params* p, uint64_t id0, int64_t n, int64_t step,
                           double* v, double* frac);

/* Tesla transformer pieces (or_tesla_* in cp_oracle.c). */
void or_tesla_matrix(const or_params* p, int coupled, double T[25]);
void or_tesla_rhs(const or_params* p, const double Qh[4][5], double c[5]);
int or_solve5(const double A[25], const double b[5], double x[5]);
/* One BDF2 step of the circuit alone (C3 an ordinary capacitor): Qh holds
   the loop charges of the last four levels (Qh[0] newest) and is shifted. */
int or_tesla_step(const or_params* p, double Qh[4][5]);
/* Loop charges Q1..Q5 of the current level of a Tesla gap. */
void or_tesla_state(const or_state* s, double Q[5]);

/* Initial plasma of n co-located electron/ion pairs at temperature T_eV
   (cell units, see or_load_pairs in cp_oracle.c). */
void or_load_pairs(const or_params* p, int64_t n, double T_eV, uint64_t seed, double* xi,
                   double* u_e, double* u_i);

/* ---- whole-gap state ---- */
or_state* or_create(const or_params* p);
void or_destroy(or_state* s);
int or_set_particles(or_state* s, int32_t species, const double* xi, const double* u,
                     const uint32_t* id, int64_t n);
int or_step(or_state* s, int32_t mode, int64_t n_steps, double tol);
int64_t or_level(const or_state* s);
int64_t or_n_live(const or_state* s, int32_t species);
int or_get_particles(const or_state* s, int32_t species, double* xi, double* u,
                     uint32_t* id, int64_t cap);
int or_read_grid(const or_state* s, double* phi, double* rho, double* E, int64_t* G);
int64_t or_history_len(const or_state* s);
int or_read_history(const or_state* s, int64_t first, int64_t n, or_diag* out);
/* Solve one coupled field problem for a given charge grid and circuit history
   without touching particles (the App. E/F validation cases). */
int or_solve_fields(const or_params* p, int32_t mode, const int64_t* G, int64_t conv_count,
                    double sigma_prev, const double* Qhist /*Q^{n-1..n-4}*/,
                    double phi0_prev /*weak: capacitor voltage handed to the circuit*/,
                    double J_hat /*weak: predicted plasma change of C phi_0 (0: plain)*/,
                    double t, double tol, double* phi, double* E,
                    double* out /*Q_n,sigma_n,I,resid*/);

/* ---- weak-coupling predictor (or_mlp.c and the learned weak mode) ----
   The weak scheme lags the strict one by J^n = C (phi_0^n - phi_0^{n-1}) -
   (Q^n - Q^{n-1}), the plasma's own change of C phi_0 over a step.  A
   40-64-64-64-2 GELU network with bfloat16 weights predicts it from the
   last 8 levels' features (Q_conv, phi_0 increment, Q_surf increment,
   secondaries emitted at x = 0, absorbed ion energy at x = 0), each divided
   by in_scale of its feature; outputs are Q_conv^{n+1}/out_scale[0]
   (auxiliary) and J^{n+1}/out_scale[1], so J_hat = out_scale[1] y[1].  The learned weak mode uses the
   prediction once 16 predictions have been checked against the realised J
   and while the running average (weight 1/16) of |J - J_hat| is at most
   bound times that of |J|; otherwise the plain lagged solve. */
#define OR_MLP_IN 40
#define OR_MLP_HIDDEN 64
#define OR_MLP_OUT 2
#define OR_MLP_NPARAM 11074
double or_bf16(float w);
double or_gelu(double x);
double or_gelu_grad(double x);
void or_mlp_forward(const float* params, int64_t n, const double* Xn, double* Yhat);
void or_mlp_loss_grad(const float* params, int64_t n, const double* Xn, const double* Yn,
                      double* grad, double* loss);
void or_adam(int64_t n, double* p, const double* g, double* m, double* v, int64_t t, double lr,
             double b1, double b2, double eps);
int or_set_predictor(or_state* s, const float* params, const double in_scale[5],
                     const double out_scale[2], double bound);

#endif
