/*
 * cp_oracle.c -- plain FP64 CPU oracle of the circuit-coupled 1D ES-PIC step
 * with ion-induced secondary electron emission (SEE).
 *
 * TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline leg (and its --impl reference arm) may load this file's
 * library; the product path never does.  It is written from the paper's
 * text, one step at a time and in the paper's order, for a reader to check
 * by eye.  Compile with -O2 -ffp-contract=off (no fused multiply-add), single
 * thread.
 *
 * Pinned by tests/test_oracle_*.py against: the closed-form series-RLC
 * response, the stationary-ion potentials of App. E.1, the printed strict
 * circuit charge of App. F, the exact uniform-field trajectory, Gauss's law
 * at both electrodes, integer charge bookkeeping, the Philox4x64-10 published
 * definition (cross-checked with numpy's independent implementation) and the
 * sample mean of the SEE yield.
 */
#include "cp_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define FIX 65536.0 /* fixed-point units per macroparticle charge on the grid */

/* ------------------------------------------------------------------------ */
/* Counter-based random numbers: Philox4x64-10 (Salmon, Moraes, Dror, Shaw,  */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11).                    */
/* ------------------------------------------------------------------------ */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

void or_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(M0, c0, &hi0, &lo0);
    mulhilo64(M1, c2, &hi1, &lo1);
    uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Top 52 bits k of a word -> open interval (0, 1): u = (k + 1/2) 2^-52, which
   is exact in binary64 (2k + 1 < 2^53), so u never rounds to 0 or 1. */
double or_u01(uint64_t w) { return ((double)(w >> 12) + 0.5) * (1.0 / 4503599627370496.0); }

/* ------------------------------------------------------------------------ */
/* Source waveform: V_s(t) = V0 (1 - cos 2 pi f t) exp(-t/tau) / 2.          */
/* ------------------------------------------------------------------------ */
double or_source(const or_params* p, double t) {
  const double pi = 3.14159265358979323846;
  return p->V0 * (1.0 - cos(2.0 * pi * p->f * t)) * exp(-t / p->tau) / 2.0;
}

/* ------------------------------------------------------------------------ */
/* Charge deposition, App. C (linear weighting) with the boundary-node rule  */
/* of App. E.2 (rho_0 = w_0 2q/dx, so no charge is lost at the wall).        */
/* Fixed point: the node weights of a particle in cell i at fraction f are   */
/* W1 = floor(f 2^16) on node i+1 and W0 = 2^16 - W1 on node i; a boundary   */
/* node receives twice its weight.  G accumulates sign(q) * weights.         */
/* ------------------------------------------------------------------------ */
void or_deposit(int64_t N, int64_t n, const double* xi, int64_t sign, int64_t* G) {
  for (int64_t p = 0; p < n; ++p) {
    double x = xi[p];
    double fl = floor(x);
    int64_t i = (int64_t)fl;
    double f = x - fl;
    int64_t W1 = (int64_t)floor(f * FIX);
    int64_t W0 = (int64_t)FIX - W1;
    if (i == 0) W0 *= 2;
    if (i + 1 == N) W1 *= 2;
    G[i] += sign * W0;
    G[i + 1] += sign * W1;
  }
}

/* ------------------------------------------------------------------------ */
/* Field gather, App. C: E_p = w_i E_{i+1/2} + w_{i+1} E_{i+3/2} from the     */
/* half-grid field; E[k] holds E_{k+1/2}, k = 0..N-1.  Between a wall and the */
/* first half-grid point the nearest edge value is used.                      */
/* ------------------------------------------------------------------------ */
double or_gather(const double* E, int64_t N, double xi) {
  if (xi < 0.5) return E[0];
  if (xi > (double)N - 0.5) return E[N - 1];
  double s = xi - 0.5;
  double js = floor(s);
  int64_t j = (int64_t)js;
  double t = s - js;
  if (j + 1 > N - 1) return E[N - 1];
  return (1.0 - t) * E[j] + t * E[j + 1];
}

/* ------------------------------------------------------------------------ */
/* Tridiagonal solve (Thomas algorithm), rows a_i x_{i-1} + b_i x_i +        */
/* c_i x_{i+1} = r_i.                                                         */
/* ------------------------------------------------------------------------ */
int or_thomas(int64_t n, const double* a, const double* b, const double* c, const double* r,
              double* x) {
  double* cp = (double*)malloc(sizeof(double) * (size_t)n);
  double* rp = (double*)malloc(sizeof(double) * (size_t)n);
  if (!cp || !rp) { free(cp); free(rp); return OR_ERR_ARG; }
  cp[0] = c[0] / b[0];
  rp[0] = r[0] / b[0];
  for (int64_t i = 1; i < n; ++i) {
    double m = b[i] - a[i] * cp[i - 1];
    cp[i] = (i + 1 < n) ? c[i] / m : 0.0;
    rp[i] = (r[i] - a[i] * rp[i - 1]) / m;
  }
  x[n - 1] = rp[n - 1];
  for (int64_t i = n - 2; i >= 0; --i) x[i] = rp[i] - cp[i] * x[i + 1];
  free(cp);
  free(rp);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* SEE sampling, Sec. 2.3 / Algorithm see_sampling_1d, with the mean yield   */
/* gamma(E) = min(scale coef sqrt(E/E_ref), gamma_max) clipped at zero and    */
/* the count floor(gamma) + Bernoulli(gamma - floor(gamma)).                  */
/* Draw 0 of (seed, SEE tag, step, ion id) decides the count.                 */
/* ------------------------------------------------------------------------ */
int64_t or_see_count(const or_params* p, double E_ion_eV, uint64_t id, int64_t step,
                     double* gamma_out) {
  double g = (p->see_scale * p->gamma_coef) * sqrt(E_ion_eV / p->E_ref_eV);
  if (g > p->gamma_max) g = p->gamma_max;
  if (!(g > 0.0)) g = 0.0;
  if (gamma_out) *gamma_out = g;
  uint64_t ctr[4] = {id, (uint64_t)step, 0, 0}, key[2] = {p->seed, OR_TAG_SEE}, w[4];
  or_philox4x64_10(ctr, key, w);
  double u1 = or_u01(w[0]);
  if (p->see_count_law == OR_SEE_COUNT_POISSON) {
    /* Algorithm see_sampling_1d: n ~ Poisson(gamma), by inversion of the
       distribution function with the same draw (the smallest n whose
       cumulative probability exceeds u1), truncated at OR_SEE_POISSON_MAX */
    double pk = exp(-g), F = pk;
    int64_t n = 0;
    while (u1 >= F && n < OR_SEE_POISSON_MAX) {
      n += 1;
      pk = pk * g / (double)n;
      F = F + pk;
    }
    return n;
  }
  double fl = floor(g);
  return (int64_t)fl + ((u1 < g - fl) ? 1 : 0);
}

/* Emitted electron j of an impact: speed from the half-Maxwellian of        */
/* temperature T_emit (|N(0,1)| times sqrt(e T / m_e), Box-Muller on draws   */
/* 0 and 1 of counter (id, step, 1 + j)), and the fraction of the step it    */
/* has already flown (draw 2).  Normal emission (Algorithm see_sampling_1d). */
void or_see_electron(const or_params* p, uint64_t id, int64_t step, int64_t j, double* v_out,
                     double* frac_out) {
  const double pi = 3.14159265358979323846;
  uint64_t ctr[4] = {id, (uint64_t)step, (uint64_t)(1 + j), 0}, key[2] = {p->seed, OR_TAG_SEE};
  uint64_t w[4];
  or_philox4x64_10(ctr, key, w);
  double ua = or_u01(w[0]), ub = or_u01(w[1]);
  double z = sqrt(-2.0 * log(ua)) * cos(2.0 * pi * ub);
  if (p->see_energy_law == OR_SEE_ENERGY_LOGNORMAL) {
    /* Algorithm see_sampling_1d: E_SE ~ Lognormal(mu, sigma), v = sqrt(2 E / m_e) */
    const double E_eV = exp(p->see_ln_mu + p->see_ln_sigma * z);
    *v_out = sqrt(2.0 * E_eV * p->e / p->m_e);
  } else {
    *v_out = sqrt(p->e * p->T_emit_eV / p->m_e) * fabs(z);
  }
  *frac_out = or_u01(w[2]);
}

void or_see_count_batch(const or_params* p, double E_ion_eV, uint64_t id0, int64_t n,
                        int64_t step, int64_t* counts) {
  for (int64_t k = 0; k < n; ++k) counts[k] = or_see_count(p, E_ion_eV, id0 + (uint64_t)k, step, NULL);
}

void or_see_electron_batch(const or_params* p, uint64_t id0, int64_t n, int64_t step, double* v,
                           double* frac) {
  for (int64_t k = 0; k < n; ++k) or_see_electron(p, id0 + (uint64_t)k, step, 0, v + k, frac + k);
}

/* ------------------------------------------------------------------------ */
/* Initial plasma: the gap starts filled with a uniform plasma of density n0  */
/* at temperature T (the paper's runs start from a loaded plasma, Sec. 3.1;  */
/* the density and temperature are the workload's).  Electrons and ions are  */
/* loaded in co-located pairs, so the initial charge density is exactly      */
/* zero.  Pair k: Philox4x64-10 counter (k, 0, 0, 0) under key (seed, load   */
/* tag); draw 0 places the pair uniformly in the gap, xi = N u0; draws 1 and */
/* 2 give a Box-Muller pair of standard normals, z_e = r cos(2 pi u2) and    */
/* z_i = r sin(2 pi u2) with r = sqrt(-2 ln u1), scaled by each species'     */
/* thermal speed sqrt(e T / m) in cells per step (a Maxwellian in 1D).        */
/* ------------------------------------------------------------------------ */
void or_load_pairs(const or_params* p, int64_t n, double T_eV, uint64_t seed, double* xi,
                   double* u_e, double* u_i) {
  const double pi = 3.14159265358979323846;
  const double Nd = (double)p->n_cells;
  const double dx = p->d / Nd;
  const double th_e = sqrt(p->e * T_eV / p->m_e) * p->dt / dx;
  const double th_i = sqrt(p->e * T_eV / p->m_i) * p->dt / dx;
  for (int64_t k = 0; k < n; ++k) {
    uint64_t ctr[4] = {(uint64_t)k, 0, 0, 0}, key[2] = {seed, OR_TAG_LOAD}, w[4];
    or_philox4x64_10(ctr, key, w);
    double x = Nd * or_u01(w[0]);
    if (x >= Nd) x = nextafter(Nd, 0.0);
    const double r = sqrt(-2.0 * log(or_u01(w[1])));
    const double a = 2.0 * pi * or_u01(w[2]);
    xi[k] = x;
    u_e[k] = th_e * (r * cos(a));
    u_i[k] = th_i * (r * sin(a));
  }
}

/* ------------------------------------------------------------------------ */
/* Tesla transformer circuit, Sec. 2.1 and App. A.  Loop equations          */
/* (Eqs. loop_1-loop_5), with X' the time derivative:                        */
/*   Q1/C1 + R1 (Q1 - Q2 - Q5)' = 0                                          */
/*   R1 (-Q1 + Q2 + Q5)' + R2 Q2' + L1 Q2'' + M Q3'' = 0                     */
/*   M Q2'' + L2 Q3'' + R3 (Q3 - Q4 + Q5)' = 0                               */
/*   R3 (-Q3 + Q4 - Q5)' + Q4/C3 = 0                                         */
/*   R1 (-Q1 + Q2 + Q5)' + Q5/C2 + R3 (Q3 - Q4 + Q5)' = 0                    */
/* BDF2 (App. A): X' = a X^n - (4 X^{n-1} - X^{n-2})/(2 dt), a = 3/(2 dt),    */
/* X'' = b X^n - (24 X^{n-1} - 22 X^{n-2} + 8 X^{n-3} - X^{n-4})/(4 dt^2),    */
/* b = 9/(4 dt^2).  The level-n terms form T Q^n, the history terms C        */
/* (derived here from the loop equations; the printed off-diagonal block and */
/* right-hand side of App. A disagree with them).  Coupled to the gap, the   */
/* load capacitor's voltage Q4/C3 is the electrode potential phi_0 (Sec.      */
/* 2.4.2): row 4 loses its 1/C3 and phi_0 moves to the right-hand side.      */
/* ------------------------------------------------------------------------ */
void or_tesla_matrix(const or_params* p, int coupled, double T[25]) {
  const double a = 3.0 / (2.0 * p->dt), b = 9.0 / (4.0 * p->dt * p->dt);
  const double r1 = a * p->tR1, r2 = a * p->tR2, r3 = a * p->tR3;
  const double m = b * p->tM;
  for (int k = 0; k < 25; ++k) T[k] = 0.0;
  /* loop 1 */
  T[0] = 1.0 / p->tC1 + r1; T[1] = -r1; T[4] = -r1;
  /* loop 2 */
  T[5] = -r1; T[6] = r1 + r2 + b * p->tL1; T[7] = m; T[9] = r1;
  /* loop 3 */
  T[11] = m; T[12] = b * p->tL2 + r3; T[13] = -r3; T[14] = r3;
  /* loop 4 */
  T[17] = -r3; T[18] = r3 + (coupled ? 0.0 : 1.0 / p->tC3); T[19] = -r3;
  /* loop 5 */
  T[20] = -r1; T[21] = r1; T[22] = r3; T[23] = -r3; T[24] = r1 + r3 + 1.0 / p->tC2;
}

/* History terms of the BDF2 loop equations: Qh[k] holds the loop charges of
   level n-1-k. */
void or_tesla_rhs(const or_params* p, const double Qh[4][5], double c[5]) {
  const double dt = p->dt;
  double h1[5], h2[5]; /* first- and second-derivative history of each loop charge */
  for (int i = 0; i < 5; ++i) {
    h1[i] = (4.0 * Qh[0][i] - Qh[1][i]) / (2.0 * dt);
    h2[i] = (24.0 * Qh[0][i] - 22.0 * Qh[1][i] + 8.0 * Qh[2][i] - Qh[3][i]) / (4.0 * dt * dt);
  }
  const double x1 = h1[0] - h1[1] - h1[4];  /* of (Q1 - Q2 - Q5), the R1 branch */
  const double x3 = h1[2] - h1[3] + h1[4];  /* of (Q3 - Q4 + Q5), the R3 branch */
  c[0] = p->tR1 * x1;
  c[1] = -p->tR1 * x1 + p->tR2 * h1[1] + p->tL1 * h2[1] + p->tM * h2[2];
  c[2] = p->tM * h2[1] + p->tL2 * h2[2] + p->tR3 * x3;
  c[3] = -p->tR3 * x3;
  c[4] = -p->tR1 * x1 + p->tR3 * x3;
}

/* Dense 5 x 5 solve, Gaussian elimination with partial pivoting. */
int or_solve5(const double A[25], const double b[5], double x[5]) {
  double M[5][6];
  for (int i = 0; i < 5; ++i) {
    for (int j = 0; j < 5; ++j) M[i][j] = A[5 * i + j];
    M[i][5] = b[i];
  }
  for (int k = 0; k < 5; ++k) {
    int piv = k;
    for (int i = k + 1; i < 5; ++i)
      if (fabs(M[i][k]) > fabs(M[piv][k])) piv = i;
    if (!(fabs(M[piv][k]) > 0.0)) return OR_ERR_ARG;
    if (piv != k)
      for (int j = 0; j < 6; ++j) { double tmp = M[k][j]; M[k][j] = M[piv][j]; M[piv][j] = tmp; }
    for (int i = k + 1; i < 5; ++i) {
      const double f = M[i][k] / M[k][k];
      for (int j = k; j < 6; ++j) M[i][j] -= f * M[k][j];
    }
  }
  for (int i = 4; i >= 0; --i) {
    double s = M[i][5];
    for (int j = i + 1; j < 5; ++j) s -= M[i][j] * x[j];
    x[i] = s / M[i][i];
  }
  return OR_OK;
}

static void shift_hist5(double Qh[4][5], const double Qn[5]) {
  for (int k = 3; k > 0; --k)
    for (int i = 0; i < 5; ++i) Qh[k][i] = Qh[k - 1][i];
  for (int i = 0; i < 5; ++i) Qh[0][i] = Qn[i];
}

int or_tesla_step(const or_params* p, double Qh[4][5]) {
  double T[25], c[5], Qn[5];
  or_tesla_matrix(p, 0, T);
  or_tesla_rhs(p, (const double(*)[5])Qh, c);
  if (or_solve5(T, c, Qn) != OR_OK) return OR_ERR_ARG;
  shift_hist5(Qh, Qn);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Coupled field solve at one time level (Sec. 2.4.2-2.4.3, App. A, App. B). */
/* ------------------------------------------------------------------------ */
typedef struct {
  double Qn, sigma_n, I, resid;
} or_solve_out;

static double row_apply(int64_t N, double b0, const double* phi, int64_t i) {
  /* (A phi)_i for the N-unknown system; phi[N] == 0 (grounded electrode). */
  if (i == 0) return b0 * phi[0] - phi[1];
  return phi[i - 1] - 2.0 * phi[i] + phi[i + 1];
}

static int solve_core(const or_params* p, int32_t mode, const int64_t* G, int64_t conv_count,
                      double sigma_prev, const double* Qh, double phi0_prev, double J_hat,
                      double t, double tol, double* phi, double* E, or_solve_out* o,
                      const double (*Qt)[5], int step_circuit, double* Qt_new) {
  const int64_t N = p->n_cells;
  const double dx = p->d / (double)N;
  const double A = p->area;
  const double eps0 = p->eps0;
  const double dt = p->dt;
  const double qw = p->e * p->weight;
  const double units = (p->grid_units > 0.0) ? p->grid_units : FIX;
  const double scale = qw / (A * dx * units); /* rho_i = G_i * scale */
  const double Qconv = (double)conv_count * qw;
  const double Vs = p->polarity * or_source(p, t);
  const double Q1 = Qh[0], Q2 = Qh[1], Q3 = Qh[2], Q4 = Qh[3];

  /* BDF2 of App. A (first and second derivative formulas) applied to the
     series loop  L Q'' + R Q' + V_gap = V_s:  a2 Q^n + a1 Q^n - hist = V_s - V_gap. */
  const double a2 = 9.0 * p->L / (4.0 * dt * dt);
  const double a1 = 3.0 * p->R / (2.0 * dt);
  const double hist = p->L * (24.0 * Q1 - 22.0 * Q2 + 8.0 * Q3 - Q4) / (4.0 * dt * dt) +
                      p->R * (4.0 * Q1 - Q2) / (2.0 * dt);
  double g = 0.0, Qpart = Q1, gam = 0.0;
  int circuit = (int)p->circuit;
  /* Tesla transformer: Q1 above is the load capacitor's loop charge Q4^{n-1} */
  double Tq[25], cq[5], uq[5], wq[5];
  const int tesla = (circuit == OR_CIRCUIT_TESLA);
  if (tesla && !Qt) return OR_ERR_ARG;
  if (tesla && step_circuit) {
    or_tesla_rhs(p, Qt, cq);
    if (mode == OR_MODE_STRICT) {
      /* Sec. 2.4.2: Q4^n = K - [T'^{-1}]_44 phi_0^n (Eqs. Q4_phi_relation, K_def) */
      const double e4[5] = {0.0, 0.0, 0.0, 1.0, 0.0};
      or_tesla_matrix(p, 1, Tq);
      if (or_solve5(Tq, cq, uq) != OR_OK || or_solve5(Tq, e4, wq) != OR_OK) return OR_ERR_ARG;
      g = wq[3];
      Qpart = uq[3]; /* K */
      gam = g * dx / (eps0 * A);
    } else {
      /* weak (Sec. 2.4.3): the circuit alone, the load capacitor's voltage
         starting from phi_0^{n-1}: loop 4 reads
         R3 (-Q3 + Q4 - Q5)' + phi_0^{n-1} + (Q4 - Q4^{n-1} + J_hat)/C3 = 0 */
      or_tesla_matrix(p, 0, Tq);
      cq[3] += -phi0_prev + (Q1 - J_hat) / p->tC3;
      if (or_solve5(Tq, cq, uq) != OR_OK) return OR_ERR_ARG;
      Qpart = uq[3];
    }
  } else if (circuit == OR_CIRCUIT_SERIES_RLC) {
    if (mode == OR_MODE_STRICT) {
      /* Eqs. Q4_phi_relation, K_def in scalar form: Q^n = K - g phi_0^n. */
      g = 1.0 / (a2 + a1);
      Qpart = g * (Vs + hist); /* K */
      gam = g * dx / (eps0 * A);
    } else {
      /* Weak mode, Sec. 2.4.3: the circuit alone is advanced one step with
         its load capacitor C, whose voltage starts from the electrode
         potential of the previous level (the capacitor state handed back
         to the circuit solver, Q_4^{n-1} = C phi_0^{n-1}); the circuit keeps
         its own loop-charge history Q.  KVL of the loop:
           a Q^n - hist + phi_0^{n-1} + (Q^n - Q^{n-1} + J_hat)/C = V_s,
         J_hat being a prediction of the plasma's own change of C phi_0 over
         the step (0 in the plain lagged scheme).  The capacitor charge
         Q*^n = C phi_0^{n-1} + Q^n - Q^{n-1} enters Eq. Poisson_BC3 against
         Q_4^{n-1} = C phi_0^{n-1}, i.e. the circuit delivers Q^n - Q^{n-1}. */
      Qpart = (Vs + hist + Q1 / p->C - phi0_prev - J_hat / p->C) / (a2 + a1 + 1.0 / p->C);
    }
  }

  /* Tridiagonal rows: row 0 is Eq. Poisson_BC2 (strict) / Poisson_BC3 (weak);
     rows 1..N-1 are Eq. dt_Poisson_app; phi_N = 0. */
  double* a = (double*)calloc((size_t)N, sizeof(double));
  double* b = (double*)calloc((size_t)N, sizeof(double));
  double* c = (double*)calloc((size_t)N, sizeof(double));
  double* r = (double*)calloc((size_t)N, sizeof(double));
  double* res = (double*)calloc((size_t)N, sizeof(double));
  double* dlt = (double*)calloc((size_t)N, sizeof(double));
  if (!a || !b || !c || !r || !res || !dlt) {
    free(a); free(b); free(c); free(r); free(res); free(dlt);
    return OR_ERR_ARG;
  }
  const double rho0 = (double)G[0] * scale;
  b[0] = 1.0 + gam;
  c[0] = -1.0;
  r[0] = (dx * dx / eps0) * ((sigma_prev + (Qconv + Qpart - Q1) / A) / dx + rho0 / 2.0);
  for (int64_t i = 1; i < N; ++i) {
    a[i] = 1.0;
    b[i] = -2.0;
    c[i] = (i + 1 < N) ? 1.0 : 0.0;
    r[i] = -dx * dx * ((double)G[i] * scale) / eps0;
  }
  or_thomas(N, a, b, c, r, phi);
  phi[N] = 0.0;

  /* Residual of all N rows plus the circuit (KVL) row, as a normwise
     backward error; iterative refinement (at most 3 sweeps) if above tol. */
  const double normA = fmax(fabs(b[0]) + 1.0, 4.0);
  double eta = 0.0;
  for (int sweep = 0; sweep <= 3; ++sweep) {
    double rmax = 0.0, pmax = 0.0, bmax = 0.0;
    for (int64_t i = 0; i < N; ++i) {
      res[i] = row_apply(N, b[0], phi, i) - r[i];
      rmax = fmax(rmax, fabs(res[i]));
      pmax = fmax(pmax, fabs(phi[i]));
      bmax = fmax(bmax, fabs(r[i]));
    }
    double den = normA * pmax + bmax;
    eta = (den > 0.0) ? rmax / den : 0.0;
    if (circuit == OR_CIRCUIT_SERIES_RLC && mode == OR_MODE_STRICT) {
      double Qn = Qpart - g * phi[0];
      double kvl = (a2 + a1) * Qn - (Vs + hist) + phi[0];
      double kden = (a2 + a1) * fabs(Qn) + fabs(Vs + hist) + fabs(phi[0]);
      if (kden > 0.0) eta = fmax(eta, fabs(kvl) / kden);
    }
    if (tesla && step_circuit && mode == OR_MODE_STRICT) {
      /* the five loop rows with Q^n = T'^{-1}(c - phi_0 e4) */
      double Qv[5];
      for (int i = 0; i < 5; ++i) Qv[i] = uq[i] - phi[0] * wq[i];
      for (int i = 0; i < 5; ++i) {
        double lhs = 0.0, den = fabs(cq[i]) + ((i == 3) ? fabs(phi[0]) : 0.0);
        for (int j = 0; j < 5; ++j) {
          lhs += Tq[5 * i + j] * Qv[j];
          den += fabs(Tq[5 * i + j] * Qv[j]);
        }
        const double ri = lhs - cq[i] + ((i == 3) ? phi[0] : 0.0);
        if (den > 0.0) eta = fmax(eta, fabs(ri) / den);
      }
    }
    if (!(eta > tol) || sweep == 3) break;
    or_thomas(N, a, b, c, res, dlt);
    for (int64_t i = 0; i < N; ++i) phi[i] -= dlt[i];
  }
  free(a); free(b); free(c); free(r); free(res); free(dlt);

  for (int64_t i = 0; i <= N; ++i)
    if (!isfinite(phi[i])) return OR_ERR_NONFINITE;

  /* Surface-charge update, Eq. top_plate_charge (Eq. sigma_update in strict
     mode).  Q^n is the circuit's loop charge in both modes; in weak mode the
     capacitor state for the next level is C phi_0^n (Sec. 2.4.3), carried as
     the level's phi_0. */
  if (tesla) {
    double Qv[5];
    for (int i = 0; i < 5; ++i)
      Qv[i] = !step_circuit ? Qt[0][i]  /* level 0: the state before the first step */
              : (mode == OR_MODE_STRICT) ? uq[i] - phi[0] * wq[i] : uq[i];
    if (Qt_new)
      for (int i = 0; i < 5; ++i) Qt_new[i] = Qv[i];
    o->Qn = Qv[3];
    o->sigma_n = sigma_prev + (Qconv + o->Qn - Q1) / A; /* Eq. sigma_update / top_plate_charge */
    o->I = (3.0 * o->Qn - 4.0 * Q1 + Q2) / (2.0 * dt);
  } else if (circuit == OR_CIRCUIT_SERIES_RLC && mode == OR_MODE_STRICT) {
    o->Qn = Qpart - g * phi[0];
    o->sigma_n = sigma_prev + (Qconv + o->Qn - Q1) / A;
    o->I = (3.0 * o->Qn - 4.0 * Q1 + Q2) / (2.0 * dt);
  } else if (circuit == OR_CIRCUIT_SERIES_RLC) {
    o->Qn = Qpart;
    o->sigma_n = sigma_prev + (Qconv + Qpart - Q1) / A;
    o->I = (3.0 * Qpart - 4.0 * Q1 + Q2) / (2.0 * dt);
  } else {
    o->sigma_n = sigma_prev + Qconv / A;
    o->Qn = Q1;
    o->I = 0.0;
  }
  /* Half-grid field, Eq. dt_E-field. */
  for (int64_t i = 0; i < N; ++i) E[i] = (phi[i] - phi[i + 1]) / dx;
  o->resid = eta;
  if (eta > tol) return OR_ERR_RESIDUAL;
  return OR_OK;
}

int or_solve_fields(const or_params* p, int32_t mode, const int64_t* G, int64_t conv_count,
                    double sigma_prev, const double* Qhist, double phi0_prev, double J_hat,
                    double t, double tol, double* phi, double* E, double* out) {
  or_solve_out o = {0, 0, 0, 0};
  if (mode == OR_MODE_WEAK_LEARNED) mode = OR_MODE_WEAK;
  int rc = solve_core(p, mode, G, conv_count, sigma_prev, Qhist, phi0_prev, J_hat, t, tol, phi,
                      E, &o, NULL, 1, NULL);
  out[0] = o.Qn;
  out[1] = o.sigma_n;
  out[2] = o.I;
  out[3] = o.resid;
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Whole-gap state and the time step.                                         */
/* ------------------------------------------------------------------------ */
struct or_state {
  or_params p;
  int64_t N;
  double dx;
  int64_t n[OR_SPECIES], cap[OR_SPECIES];
  double* xi[OR_SPECIES];
  double* u[OR_SPECIES];
  uint32_t* id; /* ions only */
  int64_t* G;   /* charge grid of the current level, N+1 nodes */
  double* phi;  /* N+1 */
  double* E;    /* N edges */
  double sigma; /* sigma_+ of the current level */
  double Qh[4]; /* Q^{n}, Q^{n-1}, Q^{n-2}, Q^{n-3} after the solve at level n */
  double Qt[4][5]; /* Tesla circuit: loop charges of levels n, n-1, n-2, n-3 */
  int64_t level;
  int solved0, pushed;
  uint64_t beam_id_base;
  /* weak-coupling predictor */
  int has_pred;
  float* pred_params;
  double in_scale[5], out_scale[2], bound;
  double feat[8][5]; /* feature rows of the last 8 levels, oldest first */
  int n_feat, pred_ready;
  double J_pred, err_avg, J_avg;
  int64_t n_eval;
  or_diag* hist;
  int64_t hist_len, hist_cap;
};

static int reserve(or_state* s, int sp, int64_t need) {
  if (need <= s->cap[sp]) return OR_OK;
  int64_t nc = s->cap[sp] ? s->cap[sp] : 1024;
  while (nc < need) nc *= 2;
  double* nx = (double*)realloc(s->xi[sp], sizeof(double) * (size_t)nc);
  if (!nx) return OR_ERR_ARG;
  s->xi[sp] = nx;
  double* nu = (double*)realloc(s->u[sp], sizeof(double) * (size_t)nc);
  if (!nu) return OR_ERR_ARG;
  s->u[sp] = nu;
  if (sp == OR_IONS) {
    uint32_t* ni = (uint32_t*)realloc(s->id, sizeof(uint32_t) * (size_t)nc);
    if (!ni) return OR_ERR_ARG;
    s->id = ni;
  }
  s->cap[sp] = nc;
  return OR_OK;
}

or_state* or_create(const or_params* p) {
  if (p->n_cells < 2 || !(p->d > 0) || !(p->area > 0) || !(p->dt > 0) || !(p->weight > 0))
    return NULL;
  or_state* s = (or_state*)calloc(1, sizeof(or_state));
  if (!s) return NULL;
  s->p = *p;
  s->N = p->n_cells;
  s->dx = p->d / (double)p->n_cells;
  s->G = (int64_t*)calloc((size_t)(s->N + 1), sizeof(int64_t));
  s->phi = (double*)calloc((size_t)(s->N + 1), sizeof(double));
  s->E = (double*)calloc((size_t)s->N, sizeof(double));
  s->sigma = p->sigma0;
  if (p->circuit == OR_CIRCUIT_TESLA) /* C1 charged, no current, before t = 0 */
    for (int k = 0; k < 4; ++k) s->Qt[k][0] = p->tC1 * p->tV1;
  return s;
}

void or_tesla_state(const or_state* s, double Q[5]) {
  for (int i = 0; i < 5; ++i) Q[i] = s->Qt[0][i];
}

void or_destroy(or_state* s) {
  if (!s) return;
  for (int sp = 0; sp < OR_SPECIES; ++sp) {
    free(s->xi[sp]);
    free(s->u[sp]);
  }
  free(s->id);
  free(s->G);
  free(s->phi);
  free(s->E);
  free(s->hist);
  free(s->pred_params);
  free(s);
}

int or_set_predictor(or_state* s, const float* params, const double in_scale[5],
                     const double out_scale[2], double bound) {
  if (!s || !params || !(bound > 0)) return OR_ERR_ARG;
  for (int f = 0; f < 5; ++f)
    if (!(in_scale[f] > 0)) return OR_ERR_ARG;
  for (int o = 0; o < 2; ++o)
    if (!(out_scale[o] > 0)) return OR_ERR_ARG;
  if (!s->pred_params) s->pred_params = (float*)malloc(sizeof(float) * OR_MLP_NPARAM);
  if (!s->pred_params) return OR_ERR_ARG;
  memcpy(s->pred_params, params, sizeof(float) * OR_MLP_NPARAM);
  memcpy(s->in_scale, in_scale, sizeof(s->in_scale));
  memcpy(s->out_scale, out_scale, sizeof(s->out_scale));
  s->bound = bound;
  s->has_pred = 1;
  return OR_OK;
}

int or_set_particles(or_state* s, int32_t sp, const double* xi, const double* u,
                     const uint32_t* id, int64_t n) {
  if (sp < 0 || sp >= OR_SPECIES || n < 0 || s->solved0) return OR_ERR_ARG;
  if (reserve(s, sp, n) != OR_OK) return OR_ERR_ARG;
  for (int64_t k = 0; k < n; ++k) {
    if (!(xi[k] > 0.0) || !(xi[k] < (double)s->N)) return OR_ERR_ARG;
    s->xi[sp][k] = xi[k];
    s->u[sp][k] = u[k];
  }
  s->n[sp] = n;
  if (sp == OR_IONS) {
    uint64_t base = 0;
    for (int64_t k = 0; k < n; ++k) {
      s->id[k] = id ? id[k] : (uint32_t)k;
      if ((uint64_t)s->id[k] + 1 > base) base = (uint64_t)s->id[k] + 1;
    }
    s->beam_id_base = base;
  }
  return OR_OK;
}

static void deposit_all(or_state* s) {
  memset(s->G, 0, sizeof(int64_t) * (size_t)(s->N + 1));
  or_deposit(s->N, s->n[OR_ELECTRONS], s->xi[OR_ELECTRONS], -1, s->G);
  or_deposit(s->N, s->n[OR_IONS], s->xi[OR_IONS], +1, s->G);
  or_deposit(s->N, s->n[OR_SECONDARIES], s->xi[OR_SECONDARIES], -1, s->G);
}

static int push_diag(or_state* s, const or_diag* d) {
  if (s->hist_len == s->hist_cap) {
    int64_t nc = s->hist_cap ? 2 * s->hist_cap : 1024;
    or_diag* nh = (or_diag*)realloc(s->hist, sizeof(or_diag) * (size_t)nc);
    if (!nh) return OR_ERR_ARG;
    s->hist = nh;
    s->hist_cap = nc;
  }
  s->hist[s->hist_len++] = *d;
  return OR_OK;
}

/* Solve at the current level and record its diagnostics row. */
static int solve_level(or_state* s, int32_t mode, double tol, int64_t conv_count, or_diag* d) {
  double Qhist[4] = {s->Qh[0], s->Qh[1], s->Qh[2], s->Qh[3]};
  or_solve_out o;
  double t = (double)s->level * s->p.dt;
  /* phi still holds the previous level (0 before the first solve: the
     circuit starts at rest) */
  const double phi0_prev = s->phi[0];
  const double sigma_prev = s->sigma;
  /* learned weak scheme: the prediction made for this level, if trusted */
  double J_used = 0.0;
  if (mode == OR_MODE_WEAK_LEARNED && s->pred_ready && s->n_eval >= 16 &&
      s->err_avg <= s->bound * s->J_avg)
    J_used = s->J_pred;
  const int32_t core_mode = (mode == OR_MODE_STRICT) ? OR_MODE_STRICT : OR_MODE_WEAK;
  double Qt_new[5] = {0, 0, 0, 0, 0};
  int rc = solve_core(&s->p, core_mode, s->G, conv_count, s->sigma, Qhist, phi0_prev, J_used, t,
                      tol, s->phi, s->E, &o, (const double(*)[5])s->Qt, s->solved0, Qt_new);
  if (rc == OR_ERR_NONFINITE || rc == OR_ERR_ARG) return rc;
  if (s->p.circuit == OR_CIRCUIT_TESLA && s->solved0) shift_hist5(s->Qt, Qt_new);
  if (s->has_pred) {
    /* the prediction for this level against the realised J */
    if (s->pred_ready) {
      const double J = s->p.C * (s->phi[0] - phi0_prev) - (o.Qn - Qhist[0]);
      s->err_avg += (fabs(J - s->J_pred) - s->err_avg) / 16.0;
      s->J_avg += (fabs(J) - s->J_avg) / 16.0;
      s->n_eval += 1;
    }
    s->pred_ready = 0;
    if (s->solved0) { /* a pushed level: append its features, predict the next */
      double row[5];
      row[0] = (double)conv_count * s->p.e * s->p.weight;
      row[1] = s->phi[0] - phi0_prev;
      row[2] = o.sigma_n * s->p.area - sigma_prev * s->p.area;
      row[3] = (double)d->emitted[0];
      row[4] = d->ion_energy_eV;
      for (int j = 0; j < 7; ++j)
        for (int f = 0; f < 5; ++f) s->feat[j][f] = s->feat[j + 1][f];
      for (int f = 0; f < 5; ++f) s->feat[7][f] = row[f];
      if (s->n_feat < 8) s->n_feat += 1;
      if (s->n_feat == 8) {
        double x[OR_MLP_IN], y[OR_MLP_OUT];
        for (int j = 0; j < 8; ++j)
          for (int f = 0; f < 5; ++f) x[5 * j + f] = s->feat[j][f] / s->in_scale[f];
        or_mlp_forward(s->pred_params, 1, x, y);
        s->J_pred = s->out_scale[1] * y[1]; /* y[0], the next Q_conv, is auxiliary */
        s->pred_ready = 1;
      }
    }
  }
  d->J_hat = J_used;
  s->sigma = o.sigma_n;
  s->Qh[3] = s->Qh[2];
  s->Qh[2] = s->Qh[1];
  s->Qh[1] = s->Qh[0];
  s->Qh[0] = o.Qn;
  d->step = s->level;
  d->t = t;
  d->V_gap = s->phi[0];
  d->I_circ = o.I;
  d->Q_surf = o.sigma_n * s->p.area;
  d->conv_count = conv_count;
  d->Q_conv = (double)conv_count * s->p.e * s->p.weight;
  d->Q_circ = o.Qn;
  d->V_source = (s->p.circuit == OR_CIRCUIT_TESLA) ? 0.0 : s->p.polarity * or_source(&s->p, t);
  d->residual = o.resid;
  for (int sp = 0; sp < OR_SPECIES; ++sp) d->n_live[sp] = s->n[sp];
  int prc = push_diag(s, d);
  return rc != OR_OK ? rc : prc;
}

static void nudge_inside(double* x, int64_t N) {
  if (*x >= (double)N) *x = nextafter((double)N, 0.0);
  if (*x <= 0.0) *x = DBL_MIN;
}

/* One leapfrog push of every live particle from level n to n+1 (Sec. 2.2.2),
   electrode absorption and ion-induced SEE (Sec. 2.3, 2.4.1), beam
   injection at x = d, and the deposit of rho^{n+1}. */
static int push_level(or_state* s, int64_t* conv_out, or_diag* d) {
  const or_params* p = &s->p;
  const int64_t N = s->N;
  const double dx = s->dx, dt = p->dt;
  const int64_t step = s->level;
  const double h = s->pushed ? 1.0 : 0.5; /* first kick: half step from v^0 */
  const double kappa[OR_SPECIES] = {-p->e * dt * dt / (p->m_e * dx),
                                    p->e * dt * dt / (p->m_i * dx),
                                    -p->e * dt * dt / (p->m_e * dx)};
  memset(d, 0, sizeof(*d));
  int64_t conv = 0, eq = 0;
  double cfl = 0.0;

  /* Emitted electrons and beam ions are collected first and appended after
     every existing particle has been pushed once. */
  int64_t se_cap = 1024, se_n = 0;
  double* se_xi = (double*)malloc(sizeof(double) * (size_t)se_cap);
  double* se_u = (double*)malloc(sizeof(double) * (size_t)se_cap);
  if (!se_xi || !se_u) { free(se_xi); free(se_u); return OR_ERR_ARG; }

  for (int sp = 0; sp < OR_SPECIES; ++sp) {
    int64_t keep = 0;
    const double kh = h * kappa[sp];
    for (int64_t k = 0; k < s->n[sp]; ++k) {
      double xi = s->xi[sp][k], u = s->u[sp][k];
      double Ep = or_gather(s->E, N, xi);
      u = u + kh * Ep;
      xi = xi + u;
      if (fabs(u) > cfl) cfl = fabs(u);
      int el = (xi <= 0.0) ? 0 : ((xi >= (double)N) ? 1 : -1);
      if (el < 0) {
        s->xi[sp][keep] = xi;
        s->u[sp][keep] = u;
        if (sp == OR_IONS) s->id[keep] = s->id[k];
        ++keep;
        continue;
      }
      /* Absorbed: convection charge at the driven electrode (Eq. for
         Q_conv^n, Sec. 2.4.1); ions trigger SEE at either electrode. */
      d->absorbed[el][sp] += 1;
      if (el == 0) conv += (sp == OR_IONS) ? 1 : -1;
      if (sp != OR_IONS) continue;
      double v = u * dx / dt;
      double Eev = 0.5 * p->m_i * v * v / p->e;
      if (el == 0) eq += llrint(Eev * 256.0);
      int64_t nse = or_see_count(p, Eev, (uint64_t)s->id[k], step, NULL);
      for (int64_t j = 0; j < nse; ++j) {
        double vse, frac;
        or_see_electron(p, (uint64_t)s->id[k], step, j, &vse, &frac);
        double use = vse * dt / dx;
        double x = (el == 0) ? use * frac : (double)N - use * frac;
        nudge_inside(&x, N);
        if (se_n == se_cap) {
          se_cap *= 2;
          se_xi = (double*)realloc(se_xi, sizeof(double) * (size_t)se_cap);
          se_u = (double*)realloc(se_u, sizeof(double) * (size_t)se_cap);
          if (!se_xi || !se_u) return OR_ERR_ARG;
        }
        se_xi[se_n] = x;
        se_u[se_n] = (el == 0) ? use : -use;
        ++se_n;
      }
      d->emitted[el] += nse;
      if (el == 0) conv += nse; /* emission removes -q_SE: + e w each */
    }
    s->n[sp] = keep;
  }

  /* Append the secondaries. */
  if (reserve(s, OR_SECONDARIES, s->n[OR_SECONDARIES] + se_n) != OR_OK) return OR_ERR_ARG;
  for (int64_t k = 0; k < se_n; ++k) {
    s->xi[OR_SECONDARIES][s->n[OR_SECONDARIES]] = se_xi[k];
    s->u[OR_SECONDARIES][s->n[OR_SECONDARIES]] = se_u[k];
    s->n[OR_SECONDARIES]++;
  }
  free(se_xi);
  free(se_u);

  /* Beam ions entering at x = d during this step: draw 0 of
     (seed, beam tag, step, k) is the fraction of the step flown, draw 1 the
     energy for a uniform spectrum. */
  const int64_t B = p->beam_per_step;
  if (B > 0) {
    if (reserve(s, OR_IONS, s->n[OR_IONS] + B) != OR_OK) return OR_ERR_ARG;
    for (int64_t k = 0; k < B; ++k) {
      uint64_t ctr[4] = {(uint64_t)k, (uint64_t)step, 0, 0}, key[2] = {p->seed, OR_TAG_BEAM};
      uint64_t w[4];
      or_philox4x64_10(ctr, key, w);
      double frac = or_u01(w[0]);
      double Eb = (p->beam_mode == 0)
                      ? p->beam_E_eV
                      : p->beam_Emin_eV + (p->beam_Emax_eV - p->beam_Emin_eV) * or_u01(w[1]);
      double v = sqrt(2.0 * Eb * p->e / p->m_i);
      double ub = v * dt / dx;
      double x = (double)N - ub * frac;
      nudge_inside(&x, N);
      int64_t q = s->n[OR_IONS]++;
      s->xi[OR_IONS][q] = x;
      s->u[OR_IONS][q] = -ub;
      s->id[q] = (uint32_t)(s->beam_id_base + (uint64_t)step * (uint64_t)B + (uint64_t)k);
    }
    d->injected = B;
  }

  deposit_all(s);
  s->pushed = 1;
  s->level += 1;
  d->max_cfl = cfl;
  d->ion_energy_eV = (double)eq / 256.0;
  *conv_out = conv;
  return OR_OK;
}

int or_step(or_state* s, int32_t mode, int64_t n_steps, double tol) {
  if (mode != OR_MODE_STRICT && mode != OR_MODE_WEAK && mode != OR_MODE_WEAK_LEARNED)
    return OR_ERR_ARG;
  if (mode == OR_MODE_WEAK_LEARNED && !s->has_pred) return OR_ERR_ARG;
  int rc = OR_OK;
  if (!s->solved0) {
    deposit_all(s);
    or_diag d;
    memset(&d, 0, sizeof(d));
    rc = solve_level(s, mode, tol, 0, &d);
    s->solved0 = 1;
    if (rc != OR_OK) return rc;
  }
  for (int64_t k = 0; k < n_steps; ++k) {
    or_diag d;
    int64_t conv = 0;
    rc = push_level(s, &conv, &d);
    if (rc != OR_OK) return rc;
    rc = solve_level(s, mode, tol, conv, &d);
    if (rc != OR_OK) return rc;
  }
  return OR_OK;
}

int64_t or_level(const or_state* s) { return s->level; }
int64_t or_n_live(const or_state* s, int32_t sp) {
  return (sp >= 0 && sp < OR_SPECIES) ? s->n[sp] : -1;
}

int or_get_particles(const or_state* s, int32_t sp, double* xi, double* u, uint32_t* id,
                     int64_t cap) {
  if (sp < 0 || sp >= OR_SPECIES || cap < s->n[sp]) return OR_ERR_ARG;
  for (int64_t k = 0; k < s->n[sp]; ++k) {
    if (xi) xi[k] = s->xi[sp][k];
    if (u) u[k] = s->u[sp][k];
    if (id && sp == OR_IONS) id[k] = s->id[k];
  }
  return OR_OK;
}

int or_read_grid(const or_state* s, double* phi, double* rho, double* E, int64_t* G) {
  const double units = (s->p.grid_units > 0.0) ? s->p.grid_units : FIX;
  const double scale = s->p.e * s->p.weight / (s->p.area * s->dx * units);
  for (int64_t i = 0; i <= s->N; ++i) {
    if (phi) phi[i] = s->phi[i];
    if (rho) rho[i] = (double)s->G[i] * scale;
    if (G) G[i] = s->G[i];
    if (E && i < s->N) E[i] = s->E[i];
  }
  return OR_OK;
}

int64_t or_history_len(const or_state* s) { return s->hist_len; }

int or_read_history(const or_state* s, int64_t first, int64_t n, or_diag* out) {
  if (first < 0 || n < 0 || first + n > s->hist_len) return OR_ERR_ARG;
  memcpy(out, s->hist + first, sizeof(or_diag) * (size_t)n);
  return OR_OK;
}
