// cp_common.cuh -- device helpers shared by the push and solve kernels.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <utility>

#include "cp_device.cuh"

namespace cg = cooperative_groups;

namespace cpk {

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

template <typename real>
struct Pair;
template <>
struct Pair<float> {
  using type = float2;
};
template <>
struct Pair<double> {
  using type = double2;
};

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

// floor(f 2^16) of a fraction f in [0, 1): exact power-of-two scaling, truncation
__device__ __forceinline__ unsigned int frac_to_fix(float f) { return __float2uint_rz(f * 65536.0f); }
__device__ __forceinline__ unsigned int frac_to_fix(double f) { return __double2uint_rz(f * 65536.0); }

// Linear interpolation between half-grid points from the pair table:
// pair j+1 = (E_{j+1/2}, E_{j+3/2} - E_{j+1/2}) with constant ends.
template <typename real>
__device__ __forceinline__ real gather(const typename Pair<real>::type* Es2, real x) {
  const real s = x - real(0.5);
  const real jf = floor(s);
  const int j = static_cast<int>(jf);
  const real t = s - jf;
  const typename Pair<real>::type e = Es2[j + 1];
  return fma(t, e.y, e.x);
}

// CIC deposit into the per-cell 32-bit sums: A[i] += 2^16 - W1 (node i),
// Bc[i] += W1 (node i+1).  Native 32-bit shared atomics.
template <typename real>
__device__ __forceinline__ void deposit(unsigned int* A, unsigned int* Bc, real x) {
  const real fl = floor(x);
  const int i = static_cast<int>(fl);
  const unsigned int w1 = frac_to_fix(x - fl);
  atomicAdd(&A[i], 65536u - w1);
  atomicAdd(&Bc[i], w1);
}

// Fold the cell sums into the int64 node grid (node k gets A[k] + Bc[k-1],
// the two end nodes doubled) and clear them.  Thread k owns node k and is
// the only reader of A[k] and Bc[k-1], so it clears exactly those.
__device__ __forceinline__ void fold(unsigned int* A, unsigned int* Bc, long long* Gs, int N,
                                     long long sign) {
  for (int k = threadIdx.x; k <= N; k += kThreads) {
    long long a = 0, b = 0;
    if (k < N) {
      a = A[k];
      A[k] = 0u;
    }
    if (k > 0) {
      b = Bc[k - 1];
      Bc[k - 1] = 0u;
    }
    if (k == 0) a <<= 1;
    if (k == N) b <<= 1;
    if (a | b) Gs[k] += sign * (a + b);
  }
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
  if (P->see_count_law == CP_SEE_COUNT_POISSON) {
    // Poisson(gamma) (Algorithm see_sampling_1d) by inversion: the smallest n
    // whose cumulative probability exceeds u1, at most kSeePoissonMax
    double pk = exp(-g), F = pk;
    int n = 0;
    while (u1 >= F && n < kSeePoissonMax) {
      n += 1;
      pk = __ddiv_rn(__dmul_rn(pk, g), static_cast<double>(n));
      F = __dadd_rn(F, pk);
    }
    return n;
  }
  const double fl = floor(g);
  return static_cast<int>(fl) + ((u1 < __dsub_rn(g, fl)) ? 1 : 0);
}

// Speed [m/s] of emitted electron j of an impact and the fraction of the step
// it has flown (draws 0, 1: Box-Muller normal z; draw 2: the fraction) of
// counter (id, step, 1 + j): |z| sqrt(e T_emit / m_e) (half-Maxwellian), or
// the lognormal law of Algorithm see_sampling_1d, E = exp(mu + sigma z) eV.
__device__ __forceinline__ double see_speed(const DevParams* P, uint64_t id, int64_t step, int j,
                                            double* frac) {
  const double pi = 3.14159265358979323846;
  const U64x4 wv = philox4x64_10(id, static_cast<uint64_t>(step), static_cast<uint64_t>(1 + j), 0,
                                 P->seed, kTagSee);
  const double ua = u01(wv.w[0]), ub = u01(wv.w[1]);
  *frac = u01(wv.w[2]);
  const double z = sqrt(-2.0 * log(ua)) * cos(2.0 * pi * ub);  // Box-Muller
  if (P->see_energy_law == CP_SEE_ENERGY_LOGNORMAL) {
    const double E_eV = exp(__dadd_rn(P->see_ln_mu, __dmul_rn(P->see_ln_sigma, z)));
    return sqrt(__ddiv_rn(__dmul_rn(__dmul_rn(2.0, E_eV), P->e), P->m_e));
  }
  return P->see_vth * fabs(z);
}

// Entry speed [cells/step] of a beam ion in the FP32 pushes (Sec. 3.2): the
// mono-energetic speed formed on the host, or sqrt(2 E e / m_i) dt / dx for
// E = E_min + (E_max - E_min) u written as sqrt(c0 + c1 u) (one FMA and one
// square root in FP64; the result is stored in FP32).
__device__ __forceinline__ double beam_speed_fp32(const DevParams* P, double u) {
  if (P->beam_mode == 0) return P->beam_ub;
  return sqrt(fma(u, P->beam_c1, P->beam_c0));
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

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) {
  return __ldcg(p);
}

__device__ __forceinline__ double source_voltage(const DevParams* P, double t) {
  const double pi = 3.14159265358979323846;
  return P->V0 * (1.0 - cos(2.0 * pi * P->f * t)) * exp(-t / P->tau) / 2.0;
}

}  // namespace cpk
