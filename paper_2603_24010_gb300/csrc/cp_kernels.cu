// cp_kernels.cu -- the fused PIC step kernel and the coupled field solve.
//
// One launch of k_step advances one time level (arXiv 2603.24010):
//   1. every CTA stages the half-grid field E^n (Epad) in shared memory and
//      streams its share of the particle store with 16-byte vector loads:
//      CIC gather (App. C), leapfrog kick and drift (Sec. 2.2.2), absorption
//      test at both electrodes (Sec. 2.4.1) and int64 fixed-point CIC
//      deposit into a shared-memory grid with the boundary-node doubling of
//      App. E.2;
//   2. each CTA then turns the ions it saw absorbed into secondary electrons
//      (Sec. 2.3, Algorithm see_sampling_1d; Philox4x64-10 draws keyed by
//      (seed, step, ion id)), appends them with warp-aggregated atomics and
//      deposits them; the CTAs also inject the beam ions of this step;
//   3. the shared-memory grids are added into the global int64 grid and the
//      per-CTA tallies into the device state;
//   4. the last CTA to finish (arrival ticket, no spinning) solves the
//      coupled Poisson/circuit system of the new level in FP64 and writes
//      E^{n+1} for the next launch (Sec. 2.4.2 strict, Sec. 2.4.3 weak).
#include <cuda_runtime.h>

#include <cstdint>

#include "cp_device.cuh"

namespace cpk {

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// ---------------------------------------------------------------------------
// 16-byte vector access to 4 consecutive particles (streaming cache hints:
// the stores are larger than L2 and touched once per step)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
  const float4 t = __ldcs(reinterpret_cast<const float4*>(p));
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void store4(float* p, const float (&v)[4]) {
  __stcs(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
}
__device__ __forceinline__ void load4(const double* p, double (&v)[4]) {
  const double2 a = __ldcs(reinterpret_cast<const double2*>(p));
  const double2 b = __ldcs(reinterpret_cast<const double2*>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void store4(double* p, const double (&v)[4]) {
  __stcs(reinterpret_cast<double2*>(p), make_double2(v[0], v[1]));
  __stcs(reinterpret_cast<double2*>(p) + 1, make_double2(v[2], v[3]));
}

__device__ __forceinline__ unsigned int frac_to_u32(float f) {
  return __float2uint_rz(f * 4294967296.0f);  // exact: power-of-two scaling of f < 1
}
__device__ __forceinline__ unsigned int frac_to_u32(double f) {
  return __double2uint_rz(f * 4294967296.0);
}

// Linear interpolation of the padded half-grid field at xi in (0, N):
// Es[j+1] = E_{j+1/2}, with Es[0] = E_{1/2} and Es[N+1] = E_{N-1/2} so that
// the field is constant between a wall and the first half-grid point.
template <typename real>
__device__ __forceinline__ real gather(const real* Es, real x) {
  const real s = x - real(0.5);
  const real jf = floor(s);
  const int j = static_cast<int>(jf);
  const real t = s - jf;
  const real e0 = Es[j + 1];
  const real e1 = Es[j + 2];
  return fma(t, e1 - e0, e0);
}

// CIC deposit in fixed point: W1 = floor(f 2^32) on node i+1, 2^32 - W1 on
// node i, boundary nodes doubled.
template <typename real>
__device__ __forceinline__ void deposit(long long* Gs, int N, real x, long long sign) {
  const real fl = floor(x);
  const int i = static_cast<int>(fl);
  const long long w1 = static_cast<long long>(frac_to_u32(x - fl));
  long long w0 = (1LL << 32) - w1;
  long long w1b = w1;
  if (i == 0) w0 <<= 1;
  if (i == N - 1) w1b <<= 1;
  atomicAdd(reinterpret_cast<unsigned long long*>(&Gs[i]),
            static_cast<unsigned long long>(sign * w0));
  atomicAdd(reinterpret_cast<unsigned long long*>(&Gs[i + 1]),
            static_cast<unsigned long long>(sign * w1b));
}

template <typename real>
__device__ __forceinline__ real nudge_inside(double x, int N) {
  real r = static_cast<real>(x);
  const real hi = nextafter(static_cast<real>(N), real(0));
  if (r >= static_cast<real>(N)) r = hi;
  if (r <= real(0)) r = (sizeof(real) == 4) ? real(1.17549435e-38f) : real(2.2250738585072014e-308);
  return r;
}

// Mean yield and count of one impact, in FP64 with every operation rounded
// as written (no contraction), so a given velocity decides the same count
// as any IEEE binary64 evaluation in the same order.
__device__ __forceinline__ int see_count(const DevParams* P, double Eev, uint64_t id, int64_t step) {
  double g = __dmul_rn(__dmul_rn(P->see_scale, P->gamma_coef),
                       __dsqrt_rn(__ddiv_rn(Eev, P->E_ref_eV)));
  if (g > P->gamma_max) g = P->gamma_max;
  if (!(g > 0.0)) g = 0.0;
  const U64x4 w = philox4x64_10(id, static_cast<uint64_t>(step), 0, 0, P->seed, kTagSee);
  const double u1 = u01(w.w[0]);
  const double fl = floor(g);
  return static_cast<int>(fl) + ((u1 < __dsub_rn(g, fl)) ? 1 : 0);
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ int warp_incl_scan(int v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, v, o);
    if (static_cast<int>(lane_id()) >= o) v += y;
  }
  return v;
}

__device__ __forceinline__ unsigned int warp_sum_u(unsigned int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned int warp_max_u(unsigned int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ---------------------------------------------------------------------------
// Block-wide scans and reductions in FP64 (one CTA, kThreads threads)
// ---------------------------------------------------------------------------
__device__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if (lane_id() == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (threadIdx.x < kThreads / 32) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  t = red[0];
  __syncthreads();
  return t;
}

__device__ double block_max(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if (lane_id() == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (threadIdx.x < kThreads / 32) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  t = red[0];
  __syncthreads();
  return t;
}

// In-place inclusive scan of a[idx(m)], m = 0..n-1, where idx(m) = m or
// n-1-m (reverse = suffix sums).  Each thread owns a contiguous run of m.
__device__ void block_incl_scan(double* a, int n, bool reverse, double* red) {
  const int per = (n + kThreads - 1) / kThreads;
  const int lo = min(static_cast<int>(threadIdx.x) * per, n);
  const int hi = min(lo + per, n);
  double s = 0.0;
  for (int m = lo; m < hi; ++m) s += a[reverse ? n - 1 - m : m];
  double incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, incl, o);
    if (static_cast<int>(lane_id()) >= o) incl += y;
  }
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if (lane_id() == 31) red[w] = incl;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = (threadIdx.x < kThreads / 32) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(0xffffffffu, t, o);
      if (static_cast<int>(threadIdx.x) >= o) t += y;
    }
    red[threadIdx.x] = t;
  }
  __syncthreads();
  double run = (w > 0 ? red[w - 1] : 0.0) + (incl - s);
  for (int m = lo; m < hi; ++m) {
    const int k = reverse ? n - 1 - m : m;
    run += a[k];
    a[k] = run;
  }
  __syncthreads();
}

// Direct solve of the N x N system with rows
//   (1 + gam) x_0 - x_1 = b_0,   x_{i-1} - 2 x_i + x_{i+1} = b_i (i >= 1), x_N = 0,
// the x = 0 Gauss row and the finite-difference Laplacian of App. B.  The
// matrix factors into two bidiagonals: with D_i = x_i - x_{i+1},
//   D_i = D_0 - sum_{j=1..i} b_j,  D_0 = b_0 - gam x_0,  x_i = sum_{k>=i} D_k,
// so x_0 (1 + N gam) = N b_0 - sum_i sum_{j=1..i} b_j.  In place: on entry
// a[i] = b_i (a[0] ignored, b_0 passed), on exit a[i] = x_i for i < N.
__device__ void tri_solve_inplace(double* a, int N, double b0, double gam, double* red,
                                  double* s_scalar) {
  if (threadIdx.x == 0) a[0] = 0.0;
  __syncthreads();
  block_incl_scan(a, N, false, red);  // a[i] = B_i = sum_{j=1..i} b_j
  double part = 0.0;
  for (int i = threadIdx.x; i < N; i += kThreads) part += a[i];
  const double T = block_sum(part, red);
  if (threadIdx.x == 0) {
    const double x0 = (static_cast<double>(N) * b0 - T) / (1.0 + static_cast<double>(N) * gam);
    s_scalar[0] = b0 - gam * x0;  // D_0
  }
  __syncthreads();
  const double D0 = s_scalar[0];
  for (int i = threadIdx.x; i < N; i += kThreads) a[i] = D0 - a[i];  // D_i
  __syncthreads();
  block_incl_scan(a, N, true, red);  // suffix sums: x_i
}

// Residual of the same system; returns the normwise backward error
// max|r| / (||A|| max|x| + max|b|) and leaves r in `r`.
__device__ double tri_residual(const double* x, const double* b, double b0, double gam, int N,
                               double* r, double* red) {
  double rm = 0.0, xm = 0.0, bm = 0.0;
  for (int i = threadIdx.x; i < N; i += kThreads) {
    const double xp = (i + 1 < N) ? x[i + 1] : 0.0;
    double ri, bi;
    if (i == 0) {
      bi = b0;
      ri = (1.0 + gam) * x[0] - xp - bi;
    } else {
      bi = b[i];
      ri = x[i - 1] - 2.0 * x[i] + xp - bi;
    }
    r[i] = ri;
    rm = fmax(rm, fabs(ri));
    xm = fmax(xm, fabs(x[i]));
    bm = fmax(bm, fabs(bi));
  }
  rm = block_max(rm, red);
  xm = block_max(xm, red);
  bm = block_max(bm, red);
  const double nA = fmax(fabs(1.0 + gam) + 1.0, 4.0);
  const double den = nA * xm + bm;
  return den > 0.0 ? rm / den : 0.0;
}

__device__ __forceinline__ double source_voltage(const DevParams* P, double t) {
  const double pi = 3.14159265358979323846;
  return P->V0 * (1.0 - cos(2.0 * pi * P->f * t)) * exp(-t / P->tau) / 2.0;
}

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) {
  return __ldcg(p);
}

// ---------------------------------------------------------------------------
// Coupled solve of the new level by the last CTA (Sec. 2.4.2 / 2.4.3).
// ---------------------------------------------------------------------------
template <typename real>
__device__ void solve_commit(const Bufs& B, int do_push, int mode, double tol,
                             unsigned char* smem) {
  const DevParams* P = B.P;
  DevState* S = B.S;
  const int N = P->N;
  double* b = reinterpret_cast<double*>(smem);  // N
  double* x = b + N;                            // N + 1
  double* w = x + (N + 1);                      // N + 1
  __shared__ double red[32];
  __shared__ double sc[24];

  const int64_t level = ldcg(&S->level) + (do_push ? 1 : 0);
  const double dt = P->dt, dx = P->dx, A = P->area, eps0 = P->eps0;
  const double qw = P->e * P->weight;
  const long long conv = do_push ? ldcg(&S->conv_count) : 0LL;

  // RHS of the Poisson rows 1..N-1 (Eq. dt_Poisson_app) and the grids
  for (int i = threadIdx.x; i <= N; i += kThreads) {
    const long long g = ldcg(&B.G[i]);
    B.Glast[i] = g;
    B.G[i] = 0;
    if (i < N) b[i] = -dx * dx * (static_cast<double>(g) * P->scale) / eps0;
  }
  if (threadIdx.x == 0) {
    const double t = static_cast<double>(level) * dt;
    const double Vs = P->polarity * source_voltage(P, t);
    const double Q1 = ldcg(&S->Qh[0]), Q2 = ldcg(&S->Qh[1]);
    const double Q3 = ldcg(&S->Qh[2]), Q4 = ldcg(&S->Qh[3]);
    const double a2 = 9.0 * P->L / (4.0 * dt * dt);
    const double a1 = 3.0 * P->R / (2.0 * dt);
    const double hist = P->L * (24.0 * Q1 - 22.0 * Q2 + 8.0 * Q3 - Q4) / (4.0 * dt * dt) +
                        P->R * (4.0 * Q1 - Q2) / (2.0 * dt);
    double g = 0.0, Qpart = Q1, gam = 0.0;
    if (P->circuit == CP_CIRCUIT_SERIES_RLC) {
      if (mode == 0) {  // strict: Q^n = K - g phi_0^n (Eqs. Q4_phi_relation, K_def)
        g = 1.0 / (a2 + a1);
        Qpart = g * (Vs + hist);
        gam = g * dx / (eps0 * A);
      } else {  // weak: free circuit with its load capacitor gives Q*^n
        Qpart = (Vs + hist) / (a2 + a1 + 1.0 / P->C);
      }
    }
    const double Qconv = static_cast<double>(conv) * qw;
    const double sigma_prev = ldcg(&S->sigma);
    const double rho0 = static_cast<double>(ldcg(&B.Glast[0])) * P->scale;
    // x = 0 row: Eq. Poisson_BC2 (strict) or Eq. Poisson_BC3 (weak)
    const double b0 = (dx * dx / eps0) * ((sigma_prev + (Qconv + Qpart - Q1) / A) / dx + rho0 / 2.0);
    sc[0] = b0; sc[1] = gam; sc[2] = g; sc[3] = Qpart; sc[4] = Vs; sc[5] = hist;
    sc[6] = a2 + a1; sc[7] = Qconv; sc[8] = sigma_prev; sc[9] = Q1; sc[10] = Q2; sc[11] = t;
    sc[12] = Q3;
  }
  __syncthreads();
  const double b0 = sc[0], gam = sc[1];
  for (int i = threadIdx.x; i < N; i += kThreads) w[i] = b[i];
  __syncthreads();
  tri_solve_inplace(w, N, b0, gam, red, sc + 16);
  for (int i = threadIdx.x; i < N; i += kThreads) x[i] = w[i];
  if (threadIdx.x == 0) x[N] = 0.0;
  __syncthreads();

  // Backward error of the Poisson rows and of the circuit row; refine.
  const bool strict_rlc = (P->circuit == CP_CIRCUIT_SERIES_RLC && mode == 0);
  double eta = 0.0;
  for (int sweep = 0; sweep <= 3; ++sweep) {
    eta = tri_residual(x, b, b0, gam, N, w, red);
    if (strict_rlc) {
      const double Qn = sc[3] - sc[2] * x[0];
      const double kvl = sc[6] * Qn - (sc[4] + sc[5]) + x[0];
      const double kden = sc[6] * fabs(Qn) + fabs(sc[4] + sc[5]) + fabs(x[0]);
      if (kden > 0.0) eta = fmax(eta, fabs(kvl) / kden);
    }
    if (!(eta > tol) || sweep == 3) break;
    const double r0 = w[0];
    __syncthreads();
    tri_solve_inplace(w, N, r0, gam, red, sc + 16);
    for (int i = threadIdx.x; i < N; i += kThreads) x[i] -= w[i];
    __syncthreads();
  }

  // Field of the new level, padded copy in particle precision.
  real* Epad = reinterpret_cast<real*>(B.Epad);
  for (int i = threadIdx.x; i < N; i += kThreads) {
    const double xp = (i + 1 < N) ? x[i + 1] : 0.0;
    const double E = (x[i] - xp) / dx;  // Eq. dt_E-field
    B.E64[i] = E;
    Epad[i + 1] = static_cast<real>(E);
    if (i == 0) Epad[0] = static_cast<real>(E);
    if (i == N - 1) Epad[N + 1] = static_cast<real>(E);
  }
  for (int i = threadIdx.x; i <= N; i += kThreads) B.phi[i] = x[i];
  __syncthreads();

  if (threadIdx.x == 0) {
    const double phi0 = x[0];
    const double Qconv = sc[7], sigma_prev = sc[8], Q1 = sc[9], Q2 = sc[10];
    double Qn, sigma_n, I;
    if (strict_rlc) {
      Qn = sc[3] - sc[2] * phi0;
      sigma_n = sigma_prev + (Qconv + Qn - Q1) / A;  // Eq. sigma_update
      I = (3.0 * Qn - 4.0 * Q1 + Q2) / (2.0 * dt);
    } else if (P->circuit == CP_CIRCUIT_SERIES_RLC) {
      sigma_n = sigma_prev + (Qconv + sc[3] - Q1) / A;  // Eq. top_plate_charge with Q*^n
      Qn = P->C * phi0;                                 // weak overwrite Q^n := C phi_0^n
      I = (3.0 * sc[3] - 4.0 * Q1 + Q2) / (2.0 * dt);
    } else {
      sigma_n = sigma_prev + Qconv / A;
      Qn = Q1;
      I = 0.0;
    }
    int status = 0;
    if (!isfinite(phi0) || !isfinite(sigma_n) || !isfinite(Qn)) status = CP_ERR_NONFINITE;
    else if (eta > tol) status = CP_ERR_RESIDUAL;

    cp_diag d;
    d.step = level;
    d.t = sc[11];
    d.V_gap = phi0;
    d.I_circ = I;
    d.Q_surf = sigma_n * A;
    d.Q_conv = Qconv;
    d.Q_circ = Qn;
    d.V_source = sc[4];
    d.residual = eta;
    d.ion_energy_eV = do_push ? static_cast<double>(ldcg(&S->ion_energy_q)) / 256.0 : 0.0;
    d.max_cfl = do_push ? static_cast<double>(__uint_as_float(ldcg(&S->max_cfl_bits))) : 0.0;
    d.pad = 0.0;
    long long nl[kSpecies];
    for (int s = 0; s < kSpecies; ++s) {
      for (int e = 0; e < 2; ++e) {
        const unsigned long long a = do_push ? ldcg(&S->absorbed[e][s]) : 0ULL;
        d.absorbed[e][s] = static_cast<int64_t>(a);
      }
      nl[s] = ldcg(&S->n_live[s]) - d.absorbed[0][s] - d.absorbed[1][s];
    }
    d.emitted[0] = do_push ? static_cast<int64_t>(ldcg(&S->emitted[0])) : 0;
    d.emitted[1] = do_push ? static_cast<int64_t>(ldcg(&S->emitted[1])) : 0;
    d.injected = do_push ? static_cast<int64_t>(ldcg(&S->injected)) : 0;
    nl[1] += d.injected;
    nl[2] += d.emitted[0] + d.emitted[1];
    for (int s = 0; s < kSpecies; ++s) d.n_live[s] = nl[s];
    d.conv_count = conv;
    S->cur = d;
    if (level < B.hist_rows) B.hist[level] = d;

    // commit the circuit and surface-charge state of the new level
    S->sigma = sigma_n;
    S->Qh[3] = sc[12];
    S->Qh[2] = Q2;
    S->Qh[1] = Q1;
    S->Qh[0] = Qn;
    S->level = level;
    if (do_push) S->pushed = 1;
    for (int s = 0; s < kSpecies; ++s) {
      S->n_live[s] = nl[s];
      for (int e = 0; e < 2; ++e) S->absorbed[e][s] = 0ULL;
    }
    S->emitted[0] = S->emitted[1] = 0ULL;
    S->injected = 0ULL;
    S->conv_count = 0;
    S->ion_energy_q = 0;
    S->max_cfl_bits = 0u;
    S->done_ctas = 0u;
    if (status != 0 && ldcg(&S->status) == 0) S->status = status;
  }
  // next push processes the slots in use, rounded up to whole vectors; the
  // padding slots are made dead here
  if (threadIdx.x < kSpecies) {
    const int s = threadIdx.x;
    long long na = static_cast<long long>(ldcg(&S->n_alloc[s]));
    if (na > P->cap[s]) na = P->cap[s];
    const long long na4 = (na + 3) & ~3LL;
    real* xs = reinterpret_cast<real*>(S->xi[s]);
    real* us = reinterpret_cast<real*>(S->u[s]);
    for (long long k = na; k < na4; ++k) {
      xs[k] = real(-1);
      us[k] = real(0);
    }
    S->n_alloc[s] = na4;
    S->n_proc[s] = na4;
  }
}

// ---------------------------------------------------------------------------
// The step kernel.
// ---------------------------------------------------------------------------
template <typename real>
__global__ void __launch_bounds__(kThreads, kCtasPerSm)
    k_step(Bufs B, int do_push, int mode, double tol) {
  const DevParams* __restrict__ P = B.P;
  DevState* S = B.S;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_abs_n;
  __shared__ int s_flag[2];  // [0]: stopped, [1]: overflow
  __shared__ unsigned long long s_cnt[2][kSpecies];
  __shared__ unsigned long long s_emit[2];
  __shared__ long long s_conv, s_energy;
  __shared__ unsigned int s_cfl, s_ticket;

  if (threadIdx.x == 0) {
    s_flag[0] = (ldcg(&S->status) != 0);
    s_flag[1] = 0;
    s_abs_n = 0;
    s_conv = 0;
    s_energy = 0;
    s_cfl = 0u;
    s_emit[0] = s_emit[1] = 0ULL;
  }
  if (threadIdx.x < 2 * kSpecies) s_cnt[threadIdx.x / kSpecies][threadIdx.x % kSpecies] = 0ULL;
  __syncthreads();
  if (s_flag[0]) return;

  const int N = P->N;
  long long* Gs = reinterpret_cast<long long*>(smem);
  real* Es = reinterpret_cast<real*>(smem + align16(sizeof(long long) * (N + 1)));
  const real* Epad = reinterpret_cast<const real*>(B.Epad);
  for (int k = threadIdx.x; k < N + 2; k += kThreads) Es[k] = Epad[k];
  for (int k = threadIdx.x; k <= N; k += kThreads) Gs[k] = 0;
  __syncthreads();

  const int64_t step = S->level;
  const bool half = (S->pushed == 0);
  const real Nr = static_cast<real>(N);
  const int cap = P->abs_cap;
  AbsRec* my_abs = B.abs + static_cast<size_t>(blockIdx.x) * cap;
  unsigned int cfl = 0u;

  for (int s = 0; s < kSpecies; ++s) {
    real* __restrict__ xs = reinterpret_cast<real*>(S->xi[s]);
    real* __restrict__ us = reinterpret_cast<real*>(S->u[s]);
    const int64_t n = S->n_proc[s];
    const long long sign = (s == CP_IONS) ? 1LL : -1LL;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kThreads * kPerThread;
    int64_t base = (static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x) * kPerThread;
    if (do_push) {
      const real kap = static_cast<real>(half ? 0.5 * P->kappa[s] : P->kappa[s]);
      const uint32_t* ids = S->id;
      unsigned int a0 = 0u, a1 = 0u;
      for (; base < n; base += stride) {
        real xv[4], uv[4];
        load4(xs + base, xv);
        load4(us + base, uv);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (xv[q] > real(0) && xv[q] < Nr) {  // live (dead slots hold -1)
            const real E = gather(Es, xv[q]);
            const real un = fma(kap, E, uv[q]);
            const real xn = xv[q] + un;
            cfl = max(cfl, __float_as_uint(fabsf(static_cast<float>(un))));
            if (!(xn > real(0) && xn < Nr)) {  // absorbed (a non-finite value counts at x = d)
              const int el = (xn <= real(0)) ? 0 : 1;
              if (el) ++a1; else ++a0;
              if (s == CP_IONS) {
                const int slot = atomicAdd(&s_abs_n, 1);
                if (slot < cap) {
                  AbsRec r;
                  r.id = ids[base + q];
                  r.electrode = static_cast<uint32_t>(el);
                  r.u = static_cast<double>(un);
                  my_abs[slot] = r;
                }
              }
              xv[q] = real(-1);
              uv[q] = real(0);
            } else {
              deposit(Gs, N, xn, sign);
              xv[q] = xn;
              uv[q] = un;
            }
          }
        }
        store4(xs + base, xv);
        store4(us + base, uv);
      }
      a0 = warp_sum_u(a0);
      a1 = warp_sum_u(a1);
      if (lane_id() == 0) {
        if (a0) atomicAdd(&s_cnt[0][s], static_cast<unsigned long long>(a0));
        if (a1) atomicAdd(&s_cnt[1][s], static_cast<unsigned long long>(a1));
      }
    } else {
      for (; base < n; base += stride) {
        real xv[4];
        load4(xs + base, xv);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (xv[q] > real(0) && xv[q] < Nr) deposit(Gs, N, xv[q], sign);
      }
    }
  }
  cfl = warp_max_u(cfl);
  if (lane_id() == 0 && cfl) atomicMax(&s_cfl, cfl);
  __syncthreads();

  if (do_push) {
    // --- secondary emission from the ions this CTA saw absorbed -----------
    const int n_abs = s_abs_n;
    if (n_abs > cap && threadIdx.x == 0) s_flag[1] = 1;
    const int na = min(n_abs, cap);
    const double dx = P->dx, dt = P->dt;
    for (int r0 = 0; r0 < na; r0 += kThreads) {
      const int r = r0 + threadIdx.x;
      const bool act = r < na;
      int nse = 0;
      AbsRec rec;
      rec.id = 0; rec.electrode = 0; rec.u = 0.0;
      if (act) {
        rec = my_abs[r];
        const double v = __ddiv_rn(__dmul_rn(rec.u, dx), dt);
        const double Eev = __ddiv_rn(__dmul_rn(__dmul_rn(__dmul_rn(0.5, P->m_i), v), v), P->e);
        nse = see_count(P, Eev, rec.id, step);
        if (rec.electrode == 0) {
          atomicAdd(reinterpret_cast<unsigned long long*>(&s_energy),
                    static_cast<unsigned long long>(__double2ll_rn(Eev * 256.0)));
          atomicAdd(reinterpret_cast<unsigned long long*>(&s_conv),
                    static_cast<unsigned long long>(static_cast<long long>(nse)));
        }
        if (nse) atomicAdd(&s_emit[rec.electrode], static_cast<unsigned long long>(nse));
      }
      const int incl = warp_incl_scan(nse);
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      unsigned long long wbase = 0ULL;
      if (lane_id() == 31 && total > 0)
        wbase = atomicAdd(reinterpret_cast<unsigned long long*>(&S->n_alloc[CP_SECONDARIES]),
                          static_cast<unsigned long long>(total));
      wbase = __shfl_sync(0xffffffffu, wbase, 31);
      if (act && nse > 0) {
        real* xs = reinterpret_cast<real*>(S->xi[CP_SECONDARIES]);
        real* us = reinterpret_cast<real*>(S->u[CP_SECONDARIES]);
        const double pi = 3.14159265358979323846;
        for (int j = 0; j < nse; ++j) {
          const U64x4 wv = philox4x64_10(rec.id, static_cast<uint64_t>(step),
                                         static_cast<uint64_t>(1 + j), 0, P->seed, kTagSee);
          const double ua = u01(wv.w[0]), ub = u01(wv.w[1]), frac = u01(wv.w[2]);
          const double z = sqrt(-2.0 * log(ua)) * cos(2.0 * pi * ub);  // Box-Muller
          const double vse = P->see_vth * fabs(z);
          const double use = vse * dt / dx;
          const double xd = (rec.electrode == 0) ? use * frac : static_cast<double>(N) - use * frac;
          const real xr = nudge_inside<real>(xd, N);
          const real ur = static_cast<real>(rec.electrode == 0 ? use : -use);
          const unsigned long long slot = wbase + static_cast<unsigned long long>(incl - nse + j);
          if (slot < static_cast<unsigned long long>(P->cap[CP_SECONDARIES])) {
            xs[slot] = xr;
            us[slot] = ur;
            deposit(Gs, N, xr, -1LL);
          } else {
            s_flag[1] = 1;
          }
        }
      }
    }

    // --- beam ions entering at x = d during this step ----------------------
    const int Bn = P->beam_per_step;
    if (Bn > 0) {
      real* xs = reinterpret_cast<real*>(S->xi[CP_IONS]);
      real* us = reinterpret_cast<real*>(S->u[CP_IONS]);
      uint32_t* ids = S->id;
      const uint32_t id0 = S->beam_id_base;
      for (int k0 = blockIdx.x * kThreads; k0 < Bn; k0 += gridDim.x * kThreads) {
        const int k = k0 + threadIdx.x;
        const bool act = k < Bn;
        const unsigned ball = __ballot_sync(0xffffffffu, act);
        unsigned long long wbase = 0ULL;
        if (lane_id() == 0 && ball)
          wbase = atomicAdd(reinterpret_cast<unsigned long long*>(&S->n_alloc[CP_IONS]),
                            static_cast<unsigned long long>(__popc(ball)));
        wbase = __shfl_sync(0xffffffffu, wbase, 0);
        if (act) {
          const U64x4 wv = philox4x64_10(static_cast<uint64_t>(k), static_cast<uint64_t>(step), 0,
                                         0, P->seed, kTagBeam);
          const double frac = u01(wv.w[0]);
          const double Eb = (P->beam_mode == 0)
                                ? P->beam_E_eV
                                : P->beam_Emin_eV + (P->beam_Emax_eV - P->beam_Emin_eV) * u01(wv.w[1]);
          const double v = sqrt(2.0 * Eb * P->e / P->m_i);
          const double ub = v * dt / dx;
          const real xr = nudge_inside<real>(static_cast<double>(N) - ub * frac, N);
          const unsigned long long slot =
              wbase + static_cast<unsigned long long>(__popc(ball & ((1u << lane_id()) - 1u)));
          if (slot < static_cast<unsigned long long>(P->cap[CP_IONS])) {
            xs[slot] = xr;
            us[slot] = static_cast<real>(-ub);
            ids[slot] = id0 + static_cast<uint32_t>(step * Bn + k);
            deposit(Gs, N, xr, 1LL);
          } else {
            s_flag[1] = 1;
          }
        }
      }
    }
  }
  __syncthreads();

  // --- add this CTA's grid and tallies into the global ones ------------------
  for (int k = threadIdx.x; k <= N; k += kThreads) {
    const long long g = Gs[k];
    if (g != 0)
      atomicAdd(reinterpret_cast<unsigned long long*>(&B.G[k]), static_cast<unsigned long long>(g));
  }
  if (threadIdx.x == 0 && do_push) {
    for (int e = 0; e < 2; ++e)
      for (int s = 0; s < kSpecies; ++s)
        if (s_cnt[e][s]) atomicAdd(&S->absorbed[e][s], s_cnt[e][s]);
    if (s_emit[0]) atomicAdd(&S->emitted[0], s_emit[0]);
    if (s_emit[1]) atomicAdd(&S->emitted[1], s_emit[1]);
    // convection count at x = 0: ions - electrons absorbed + secondaries emitted
    const long long conv = static_cast<long long>(s_cnt[0][CP_IONS]) -
                           static_cast<long long>(s_cnt[0][CP_ELECTRONS]) -
                           static_cast<long long>(s_cnt[0][CP_SECONDARIES]) + s_conv;
    if (conv) atomicAdd(reinterpret_cast<unsigned long long*>(&S->conv_count),
                        static_cast<unsigned long long>(conv));
    if (s_energy) atomicAdd(reinterpret_cast<unsigned long long*>(&S->ion_energy_q),
                            static_cast<unsigned long long>(s_energy));
    if (s_cfl) atomicMax(&S->max_cfl_bits, s_cfl);
    if (blockIdx.x == 0 && P->beam_per_step > 0)
      atomicAdd(&S->injected, static_cast<unsigned long long>(P->beam_per_step));
    if (s_flag[1]) atomicCAS(&S->status, 0, CP_ERR_CAPACITY);
  }

  // --- the last CTA to arrive solves the new level ---------------------------
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_ticket = atomicAdd(&S->done_ctas, 1u);
  __syncthreads();
  if (s_ticket != gridDim.x - 1) return;
  __threadfence();
  solve_commit<real>(B, do_push, mode, tol, smem);
}

// ---------------------------------------------------------------------------
// Removal of absorbed particles: live slots are packed into the spare buffer
// (warp-contiguous, order not kept) and the buffers are swapped by the last
// CTA.  Physics does not depend on particle order.
// ---------------------------------------------------------------------------
template <typename real>
__global__ void __launch_bounds__(kThreads) k_compact(Bufs B) {
  const DevParams* __restrict__ P = B.P;
  DevState* S = B.S;
  __shared__ unsigned int s_ticket;
  __shared__ int s_stop;
  if (threadIdx.x == 0) s_stop = (ldcg(&S->status) != 0);
  __syncthreads();
  if (s_stop) return;
  for (int s = 0; s < kSpecies; ++s) {
    const real* xs = reinterpret_cast<const real*>(S->xi[s]);
    const real* us = reinterpret_cast<const real*>(S->u[s]);
    real* xd = reinterpret_cast<real*>(S->xi_alt[s]);
    real* ud = reinterpret_cast<real*>(S->u_alt[s]);
    const uint32_t* is = S->id;
    uint32_t* id_d = S->id_alt;
    const int64_t n = S->n_proc[s];
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kThreads * kPerThread;
    // uniform trip count so that every warp stays converged for the shuffles
    const int64_t trips = (n + stride - 1) / stride;
    for (int64_t t = 0; t < trips; ++t) {
      const int64_t base =
          t * stride + (static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x) * kPerThread;
      real xv[4] = {real(-1), real(-1), real(-1), real(-1)}, uv[4] = {0, 0, 0, 0};
      if (base < n) {
        load4(xs + base, xv);
        load4(us + base, uv);
      }
      int c = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) c += (xv[q] > real(0)) ? 1 : 0;
      const int incl = warp_incl_scan(c);
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      unsigned long long wb = 0ULL;
      if (lane_id() == 31 && total > 0) wb = atomicAdd(&S->compact_n[s], static_cast<unsigned long long>(total));
      wb = __shfl_sync(0xffffffffu, wb, 31);
      unsigned long long o = wb + static_cast<unsigned long long>(incl - c);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (xv[q] > real(0)) {
          xd[o] = xv[q];
          ud[o] = uv[q];
          if (s == CP_IONS) id_d[o] = is[base + q];
          ++o;
        }
      }
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_ticket = atomicAdd(&S->compact_done, 1u);
  __syncthreads();
  if (s_ticket != gridDim.x - 1) return;
  __threadfence();
  if (threadIdx.x < kSpecies) {
    const int s = threadIdx.x;
    const long long cnt = static_cast<long long>(ldcg(&S->compact_n[s]));
    const long long c4 = (cnt + 3) & ~3LL;
    real* xd = reinterpret_cast<real*>(S->xi_alt[s]);
    real* ud = reinterpret_cast<real*>(S->u_alt[s]);
    for (long long k = cnt; k < c4; ++k) {
      xd[k] = real(-1);
      ud[k] = real(0);
    }
    void* t0 = S->xi[s];
    S->xi[s] = S->xi_alt[s];
    S->xi_alt[s] = t0;
    void* t1 = S->u[s];
    S->u[s] = S->u_alt[s];
    S->u_alt[s] = t1;
    S->n_alloc[s] = c4;
    S->n_proc[s] = c4;
    S->compact_n[s] = 0ULL;
  }
  if (threadIdx.x == 0) {
    uint32_t* t2 = S->id;
    S->id = S->id_alt;
    S->id_alt = t2;
    S->compact_done = 0u;
  }
}

template <typename real>
__global__ void k_fill(real* p, int64_t n, real v) {
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    p[i] = v;
}

// ---------------------------------------------------------------------------
// Host-side launchers (internal C++ interface used by cp_api.cu)
// ---------------------------------------------------------------------------
size_t step_smem_bytes(int N, int precision) {
  const size_t es = (precision == CP_FP32) ? sizeof(float) : sizeof(double);
  const size_t particle = align16(sizeof(long long) * (N + 1)) + es * (N + 2);
  const size_t solve = sizeof(double) * (3 * static_cast<size_t>(N) + 2);
  return particle > solve ? particle : solve;
}

cudaError_t step_configure(int precision, size_t smem) {
  if (precision == CP_FP32)
    return cudaFuncSetAttribute(k_step<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(smem));
  return cudaFuncSetAttribute(k_step<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(smem));
}

cudaError_t step_occupancy(int precision, size_t smem, int* blocks_per_sm) {
  if (precision == CP_FP32)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_step<float>, kThreads, smem);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_step<double>, kThreads, smem);
}

cudaError_t step_launch(int precision, const Bufs& B, int grid, size_t smem, cudaStream_t st,
                        int do_push, int mode, double tol) {
  if (precision == CP_FP32)
    k_step<float><<<grid, kThreads, smem, st>>>(B, do_push, mode, tol);
  else
    k_step<double><<<grid, kThreads, smem, st>>>(B, do_push, mode, tol);
  return cudaGetLastError();
}

cudaError_t compact_launch(int precision, const Bufs& B, int grid, cudaStream_t st) {
  if (precision == CP_FP32)
    k_compact<float><<<grid, kThreads, 0, st>>>(B);
  else
    k_compact<double><<<grid, kThreads, 0, st>>>(B);
  return cudaGetLastError();
}

cudaError_t fill_launch(int precision, void* p, int64_t n, double v, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = static_cast<int>((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  if (precision == CP_FP32)
    k_fill<float><<<grid, 256, 0, st>>>(reinterpret_cast<float*>(p), n, static_cast<float>(v));
  else
    k_fill<double><<<grid, 256, 0, st>>>(reinterpret_cast<double*>(p), n, v);
  return cudaGetLastError();
}

}  // namespace cpk
