// cp_push.cu -- the particle push of the PIC step, the removal of absorbed
// particles, and small set-up kernels.
//
// One time step (arXiv 2603.24010) is two launches, this push and the
// cluster solve of cp_solve.cu.
//
// k_push  (persistent grid, 2 CTAs per SM) streams every particle once with
//   16-byte vector loads/stores: CIC gather of E^n from a shared-memory
//   table (App. C), leapfrog kick and drift (Sec. 2.2.2), absorption at the
//   electrodes (Sec. 2.4.1), and the CIC deposit of rho^{n+1} in fixed point
//   (2^16 units per macroparticle charge, boundary nodes doubled as in
//   App. E.2) into per-cell 32-bit shared-memory sums that are folded into a
//   shared int64 node grid every 31 tiles (so no 32-bit sum can overflow).
//   Each CTA then turns the ions it saw absorbed into secondary electrons
//   (Sec. 2.3, Algorithm see_sampling_1d; Philox4x64-10 draws keyed by
//   (seed, step, ion id)), appends them with warp-aggregated atomics and
//   deposits them; the CTAs share the injection of the step's beam ions.
//   The int64 node grids and the tallies are added into global memory.
//
// k_compact packs the live particles of every species into the spare
//   buffers every few steps (dead slots are skipped by the push until then).
#include "cp_common.cuh"

namespace cpk {
// ---------------------------------------------------------------------------
// k_push
// ---------------------------------------------------------------------------
template <typename real>
__global__ void __launch_bounds__(kThreads, kCtasPerSm) k_push(Bufs B, int do_push) {
  using real2 = typename Pair<real>::type;
  const DevParams* __restrict__ P = B.P;
  DevState* S = B.S;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_abs_n;
  __shared__ int s_flag[2];  // [0]: stopped, [1]: overflow
  __shared__ unsigned long long s_cnt[2][kSpecies];
  __shared__ unsigned long long s_emit[2];
  __shared__ long long s_conv, s_energy;
  __shared__ unsigned int s_cfl;

  cudaGridDependencySynchronize();  // the previous solve (or removal) has completed
  cudaTriggerProgrammaticLaunchCompletion();
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
  const int64_t step = S->level;

  long long* Gs = reinterpret_cast<long long*>(smem);
  unsigned int* A = reinterpret_cast<unsigned int*>(smem + align16(sizeof(long long) * (N + 1)));
  unsigned int* Bc = A + N;
  real2* Es2 = reinterpret_cast<real2*>(smem + align16(sizeof(long long) * (N + 1)) +
                                        align16(sizeof(unsigned int) * 2 * N));
  const real2* Epair = reinterpret_cast<const real2*>(B.Epair);
  for (int k = threadIdx.x; k <= N; k += kThreads) {
    Es2[k] = Epair[k];
    Gs[k] = 0;
  }
  for (int k = threadIdx.x; k < 2 * N; k += kThreads) A[k] = 0u;
  __syncthreads();

  const bool half = (S->pushed == 0);
  const real Nr = static_cast<real>(N);
  const int cap = P->abs_cap;
  AbsRec* my_abs = B.abs + static_cast<size_t>(blockIdx.x) * cap;
  unsigned int cfl = 0u;

  for (int s = 0; s < kSpecies; ++s) {
    real* __restrict__ xs = reinterpret_cast<real*>(S->xi[s]);
    real* __restrict__ us = reinterpret_cast<real*>(S->u[s]);
    const int64_t n = S->n_proc[s];  // multiple of 4
    const int64_t ntiles = (n + kTile - 1) / kTile;
    const long long sign = (s == CP_IONS) ? 1LL : -1LL;
    real kap;
    if constexpr (sizeof(real) == 4) kap = P->kap_f[half ? 0 : 1][s];
    else kap = P->kap_d[half ? 0 : 1][s];
    const uint32_t* ids = S->id;
    unsigned int a0 = 0u, a1 = 0u;
    int since = 0;
    // two tiles in flight per thread: the next tile's loads are issued
    // before the current tile is processed
    real xv[4], uv[4];
    int64_t base = static_cast<int64_t>(blockIdx.x) * kTile + static_cast<int64_t>(threadIdx.x) * kPerThread;
    if (base < n) {
      load4(xs + base, xv);
      if (do_push) load4(us + base, uv);
    }
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int64_t bnext = base + static_cast<int64_t>(gridDim.x) * kTile;
      real xq[4], uq[4];
      const bool more = bnext < n;
      if (more) {
        load4(xs + bnext, xq);
        if (do_push) load4(us + bnext, uq);
      }
      if (base < n) {
        if (do_push) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (xv[q] > real(0) && xv[q] < Nr) {  // live (dead slots hold -1)
              const real E = gather<real>(Es2, xv[q]);
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
                deposit<real>(A, Bc, xn);
                xv[q] = xn;
                uv[q] = un;
              }
            }
          }
          store4(xs + base, xv);
          store4(us + base, uv);
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (xv[q] > real(0) && xv[q] < Nr) deposit<real>(A, Bc, xv[q]);
        }
      }
      if (more) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          xv[q] = xq[q];
          uv[q] = uq[q];
        }
      }
      base = bnext;
      if (++since == kFlushTiles) {  // bounds every 32-bit cell sum below 2^32
        __syncthreads();
        fold(A, Bc, Gs, N, sign);
        __syncthreads();
        since = 0;
      }
    }
    __syncthreads();
    fold(A, Bc, Gs, N, sign);
    __syncthreads();
    a0 = warp_sum_u(a0);
    a1 = warp_sum_u(a1);
    if (lane_id() == 0) {
      if (a0) atomicAdd(&s_cnt[0][s], static_cast<unsigned long long>(a0));
      if (a1) atomicAdd(&s_cnt[1][s], static_cast<unsigned long long>(a1));
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
        for (int j = 0; j < nse; ++j) {
          double frac;
          const double vse = see_speed(P, rec.id, step, j, &frac);
          const double use = vse * dt / dx;
          const double xd = (rec.electrode == 0) ? __dmul_rn(use, frac) : __dsub_rn(static_cast<double>(N), __dmul_rn(use, frac));
          const real xr = nudge_inside<real>(xd, N);
          const real ur = static_cast<real>(rec.electrode == 0 ? use : -use);
          const unsigned long long slot = wbase + static_cast<unsigned long long>(incl - nse + j);
          if (slot < static_cast<unsigned long long>(P->cap[CP_SECONDARIES])) {
            xs[slot] = xr;
            us[slot] = ur;
            deposit<real>(A, Bc, xr);
          } else {
            s_flag[1] = 1;
          }
        }
      }
      if (P->see_count_law == CP_SEE_COUNT_POISSON) {  // up to 512 x 64 electrons per round
        __syncthreads();
        fold(A, Bc, Gs, N, -1LL);
        __syncthreads();
      }
    }
    __syncthreads();
    if (na > 0) {  // floor + Bernoulli: at most 4096 impacts x 15 electrons, no 32-bit overflow
      fold(A, Bc, Gs, N, -1LL);
      __syncthreads();
    }

    // --- beam ions entering at x = d during this step ----------------------
    const int Bn = P->beam_per_step;
    if (Bn > 0 && static_cast<int>(blockIdx.x) * kThreads < Bn) {
      real* xs = reinterpret_cast<real*>(S->xi[CP_IONS]);
      real* us = reinterpret_cast<real*>(S->u[CP_IONS]);
      uint32_t* ids = S->id;
      const uint32_t id0 = S->beam_id_base;
      int since = 0;
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
                                : __dadd_rn(P->beam_Emin_eV, __dmul_rn(__dsub_rn(P->beam_Emax_eV, P->beam_Emin_eV), u01(wv.w[1])));
          const double v = sqrt(2.0 * Eb * P->e / P->m_i);
          const double ub = v * dt / dx;
          const real xr = nudge_inside<real>(__dsub_rn(static_cast<double>(N), __dmul_rn(ub, frac)), N);
          const unsigned long long slot =
              wbase + static_cast<unsigned long long>(__popc(ball & ((1u << lane_id()) - 1u)));
          if (slot < static_cast<unsigned long long>(P->cap[CP_IONS])) {
            xs[slot] = xr;
            us[slot] = static_cast<real>(-ub);
            ids[slot] = id0 + static_cast<uint32_t>(step * Bn + k);
            deposit<real>(A, Bc, xr);
          } else {
            s_flag[1] = 1;
          }
        }
        if (++since == 4 * kFlushTiles) {  // 512 ions per pass: bounded cell sums
          __syncthreads();
          fold(A, Bc, Gs, N, 1LL);
          __syncthreads();
          since = 0;
        }
      }
      __syncthreads();
      fold(A, Bc, Gs, N, 1LL);
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
}

// ---------------------------------------------------------------------------
// Removal of absorbed particles: live slots are packed into the spare buffer
// (warp-contiguous, order not kept) and the buffers are swapped by the last
// CTA.  Physics does not depend on particle order.
// ---------------------------------------------------------------------------
template <typename real>
__global__ void __launch_bounds__(kThreads) k_compact(Bufs B) {
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

// polarity V_s(t_n) for n = 0..rows-1, once at set-up (the source of Sec. 2.1)
__global__ void k_source_table(const DevParams* P, double* vs, int64_t rows) {
  for (int64_t n = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; n < rows;
       n += static_cast<int64_t>(gridDim.x) * blockDim.x)
    vs[n] = P->polarity * source_voltage(P, static_cast<double>(n) * P->dt);
}

cudaError_t source_table_launch(const DevParams* P, double* vs, int64_t rows, cudaStream_t st) {
  const int grid = static_cast<int>((rows + 255) / 256 < 1024 ? (rows + 255) / 256 : 1024);
  k_source_table<<<grid, 256, 0, st>>>(P, vs, rows);
  return cudaGetLastError();
}

// Initial plasma: n co-located electron/ion pairs at temperature T (the
// paper's runs start from a loaded plasma, Sec. 3.1).  Pair k draws
// Philox4x64-10 counter (k, 0, 0, 0) under key (seed, load tag): xi = N u0
// (uniform in the gap), and the Box-Muller pair of u1, u2 gives the two
// velocities, z_e th_e and z_i th_i (th = sqrt(e T / m) dt / dx, a 1D
// Maxwellian).  Positions are rounded to the store's precision and kept
// inside (0, N); ion ids are k.
template <typename real>
__global__ void k_load_pairs(real* xe, real* ue, real* xo, real* uo, uint32_t* id, int64_t n, int N,
                             double th_e, double th_i, uint64_t seed) {
  const double pi = 3.14159265358979323846;
  for (int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < n;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const U64x4 w = philox4x64_10(static_cast<uint64_t>(k), 0, 0, 0, seed, kTagLoad);
    const real x = nudge_inside<real>(__dmul_rn(static_cast<double>(N), u01(w.w[0])), N);
    const double r = sqrt(-2.0 * log(u01(w.w[1])));
    const double a = __dmul_rn(2.0 * pi, u01(w.w[2]));
    xe[k] = x;
    xo[k] = x;
    ue[k] = static_cast<real>(__dmul_rn(th_e, __dmul_rn(r, cos(a))));
    uo[k] = static_cast<real>(__dmul_rn(th_i, __dmul_rn(r, sin(a))));
    id[k] = static_cast<uint32_t>(k);
  }
}

cudaError_t load_pairs_launch(int precision, void* xe, void* ue, void* xo, void* uo, uint32_t* id,
                              int64_t n, int N, double th_e, double th_i, uint64_t seed, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int grid = static_cast<int>((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192);
  if (precision == CP_FP32)
    k_load_pairs<float><<<grid, 256, 0, st>>>(static_cast<float*>(xe), static_cast<float*>(ue),
                                              static_cast<float*>(xo), static_cast<float*>(uo), id, n, N,
                                              th_e, th_i, seed);
  else
    k_load_pairs<double><<<grid, 256, 0, st>>>(static_cast<double*>(xe), static_cast<double*>(ue),
                                               static_cast<double*>(xo), static_cast<double*>(uo), id, n,
                                               N, th_e, th_i, seed);
  return cudaGetLastError();
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
// FP32 particles take the push of cp_push_async.cu.
size_t push_async_smem_bytes(int N);
cudaError_t push_async_configure(size_t smem);
cudaError_t push_async_occupancy(size_t smem, int* blocks_per_sm);
cudaError_t push_async_launch(const Bufs& B, int grid, size_t smem, cudaStream_t st, int do_push);

cudaError_t push_configure(int precision, size_t push_smem) {
  if (precision == CP_FP32) return push_async_configure(push_smem);
  return cudaFuncSetAttribute(k_push<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(push_smem));
}

size_t push_smem_bytes(int N, int precision) {
  if (precision == CP_FP32) return push_async_smem_bytes(N);
  const size_t es = (precision == CP_FP32) ? sizeof(float) : sizeof(double);
  return align16(sizeof(long long) * (N + 1)) + align16(sizeof(unsigned int) * 2 * N) +
         2 * es * (N + 1);
}

cudaError_t push_occupancy(int precision, size_t smem, int* blocks_per_sm) {
  if (precision == CP_FP32) return push_async_occupancy(smem, blocks_per_sm);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_push<double>, kThreads, smem);
}

// Push and solve are launched with programmatic dependent launch: each may
// be scheduled while its predecessor finishes and waits in
// cudaGridDependencySynchronize() until that grid has completed.
cudaError_t push_launch(int precision, const Bufs& B, int grid, size_t smem, cudaStream_t st,
                        int do_push) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (precision == CP_FP32) return push_async_launch(B, grid, smem, st, do_push);
  return cudaLaunchKernelEx(&cfg, k_push<double>, B, do_push);
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
