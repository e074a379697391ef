// cp_batch.cu -- the ensemble path: many independent gap instances advanced
// by one persistent launch per stage.
//
// k_push_ens: the particle tiles of every (instance, species) pair form one
//   flat work list (instance-major, then species, then tile); each CTA takes
//   one contiguous share of it, so it meets only a few instances and loads
//   each instance's gather table and flushes each instance's deposit grid
//   once per step.  Per tile the arithmetic is that of the single-instance
//   push (same gather, kick, drift, absorption test and fixed-point deposit),
//   so an instance advanced in the ensemble follows exactly the trajectory
//   it follows alone.  Secondary emission and the beam are handled after the
//   tiles: emitted electrons and beam ions are deposited with int64 global
//   atomics straight into their instance's grid.
// k_compact_ens / k_swap_ens: removal of absorbed particles over the same
//   flat list, then one thread per (instance, species) swaps the buffers.
// The solve of every instance (one CTA each) is k_solve_ens in cp_solve.cu.
#include "cp_common.cuh"

namespace cpk {

// Absorbed ion of the ensemble push: instance and electrode packed.
struct AbsRecE {
  uint32_t id;
  uint32_t inst_el;  // instance * 2 + electrode
  double u;
};

constexpr int kEnsMaxEntries = 3 * 2048;  // (instance, species) pairs: at most 2048 instances

__device__ __forceinline__ void fold_any(unsigned int* A, unsigned int* Bc, long long* Gs, int N,
                                         long long sign) {
  for (int k = threadIdx.x; k <= N; k += blockDim.x) {
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

// The fixed-point CIC deposit of one particle, added straight into an int64
// global grid (end nodes doubled, as the fold does).
template <typename real>
__device__ __forceinline__ void deposit_global(long long* G, int N, real x, long long sign) {
  const real fl = floor(x);
  const int i = static_cast<int>(fl);
  const long long w1 = static_cast<long long>(frac_to_fix(x - fl));
  const long long w0 = 65536LL - w1;
  atomicAdd(reinterpret_cast<unsigned long long*>(&G[i]),
            static_cast<unsigned long long>(sign * (i == 0 ? 2 * w0 : w0)));
  atomicAdd(reinterpret_cast<unsigned long long*>(&G[i + 1]),
            static_cast<unsigned long long>(sign * (i + 1 == N ? 2 * w1 : w1)));
}

// Exclusive prefix of the tile counts of every (instance, species) pair into
// off[0..n] (off[n] = total); counts of stopped instances are 0.
template <int THREADS>
__device__ void tile_offsets(const Bufs* __restrict__ Ball, int E, int tile, int* off, int* wsum) {
  const int n = 3 * E;
  const int per = (n + THREADS - 1) / THREADS;
  const int j0 = min(static_cast<int>(threadIdx.x) * per, n), j1 = min(j0 + per, n);
  int loc = 0;
  for (int j = j0; j < j1; ++j) {
    const DevState* S = Ball[j / 3].S;
    const long long np = (ldcg(&S->status) == 0) ? ldcg(&S->n_proc[j % 3]) : 0LL;
    const int t = static_cast<int>((np + tile - 1) / tile);
    off[j] = t;
    loc += t;
  }
  // block exclusive scan of the per-thread sums
  int incl = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (static_cast<int>(lane_id()) >= o) incl += y;
  }
  const int w = threadIdx.x >> 5;
  if (lane_id() == 31) wsum[w] = incl;
  __syncthreads();
  int wbase = 0;
  for (int q = 0; q < w; ++q) wbase += wsum[q];
  int run = wbase + incl - loc;
  for (int j = j0; j < j1; ++j) {
    const int t = off[j];
    off[j] = run;
    run += t;
  }
  if (threadIdx.x == THREADS - 1) off[n] = wbase + incl;
  __syncthreads();
}

template <typename real, int THREADS>
__global__ void __launch_bounds__(THREADS)
k_push_ens(const Bufs* __restrict__ Ball, int E, int n_max, AbsRecE* __restrict__ abs_all, int abs_cap) {
  using real2 = typename Pair<real>::type;
  constexpr int TILE = THREADS * kPerThread;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int wsum[THREADS / 32];
  __shared__ int s_abs_n, s_j;
  __shared__ unsigned long long s_cnt[2][kSpecies];
  __shared__ unsigned int s_cfl;

  cudaGridDependencySynchronize();  // the previous solves (or removal) have completed
  cudaTriggerProgrammaticLaunchCompletion();
  long long* Gs = reinterpret_cast<long long*>(smem);
  unsigned int* A = reinterpret_cast<unsigned int*>(smem + align16(sizeof(long long) * (n_max + 1)));
  unsigned int* Bc = A + n_max;
  real2* Es2 = reinterpret_cast<real2*>(smem + align16(sizeof(long long) * (n_max + 1)) +
                                        align16(sizeof(unsigned int) * 2 * n_max));
  int* off = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(Es2) +
                                    align16(sizeof(real2) * (n_max + 1)));
  tile_offsets<THREADS>(Ball, E, TILE, off, wsum);
  const long long U = off[3 * E];
  const long long u0 = U * blockIdx.x / gridDim.x, u1 = U * (blockIdx.x + 1) / gridDim.x;
  if (threadIdx.x == 0) {
    s_abs_n = 0;
    int lo = 0, hi = 3 * E;  // the entry holding unit u0: off[j] <= u0 < off[j+1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (off[mid] <= u0) lo = mid;
      else hi = mid;
    }
    s_j = lo;
  }
  for (int k = threadIdx.x; k <= n_max; k += THREADS) Gs[k] = 0;
  for (int k = threadIdx.x; k < 2 * n_max; k += THREADS) A[k] = 0u;
  __syncthreads();
  AbsRecE* my_abs = abs_all + static_cast<size_t>(blockIdx.x) * abs_cap;

  int cur = -1, N = 0;
  const DevParams* P = nullptr;
  DevState* S = nullptr;
  bool half = false;
  unsigned int cfl = 0u;
  // flush the current instance's grid and tallies into global memory
  auto flush = [&]() {
    __syncthreads();
    long long* G = Ball[cur].G;
    for (int k = threadIdx.x; k <= N; k += THREADS) {
      const long long g = Gs[k];
      if (g != 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&G[k]), static_cast<unsigned long long>(g));
        Gs[k] = 0;
      }
    }
    const unsigned int c = warp_max_u(cfl);
    if (lane_id() == 0 && c) atomicMax(&S->max_cfl_bits, c);
    cfl = 0u;
    if (threadIdx.x == 0) {
      for (int e = 0; e < 2; ++e)
        for (int s = 0; s < kSpecies; ++s)
          if (s_cnt[e][s]) atomicAdd(&S->absorbed[e][s], s_cnt[e][s]);
      const long long conv = static_cast<long long>(s_cnt[0][CP_IONS]) -
                             static_cast<long long>(s_cnt[0][CP_ELECTRONS]) -
                             static_cast<long long>(s_cnt[0][CP_SECONDARIES]);
      if (conv) atomicAdd(reinterpret_cast<unsigned long long*>(&S->conv_count),
                          static_cast<unsigned long long>(conv));
    }
    __syncthreads();
  };

  for (long long u = u0; u < u1;) {
    const int j = s_j;
    const int inst = j / 3, s = j % 3;
    const long long t_end = min(u1, static_cast<long long>(off[j + 1]));
    const long long t0 = u - off[j], t1 = t_end - off[j];  // tiles of this (instance, species)
    if (inst != cur) {
      if (cur >= 0) flush();
      cur = inst;
      const Bufs& B = Ball[cur];
      P = B.P;
      S = B.S;
      N = P->N;
      half = (ldcg(&S->pushed) == 0);
      const real2* Epair = reinterpret_cast<const real2*>(B.Epair);
      for (int k = threadIdx.x; k <= N; k += THREADS) Es2[k] = Epair[k];
      if (threadIdx.x < 2 * kSpecies) s_cnt[threadIdx.x / kSpecies][threadIdx.x % kSpecies] = 0ULL;
      if (threadIdx.x == 0) s_cfl = 0u;
      __syncthreads();
    }
    real* __restrict__ xs = reinterpret_cast<real*>(S->xi[s]);
    real* __restrict__ us = reinterpret_cast<real*>(S->u[s]);
    const int64_t n = S->n_proc[s];
    const long long sign = (s == CP_IONS) ? 1LL : -1LL;
    real kap;
    if constexpr (sizeof(real) == 4) kap = P->kap_f[half ? 0 : 1][s];
    else kap = P->kap_d[half ? 0 : 1][s];
    const real Nr = static_cast<real>(N);
    const uint32_t* ids = S->id;
    unsigned int a0 = 0u, a1 = 0u;
    int since = 0;
    real xv[4], uv[4];
    int64_t base = t0 * TILE + static_cast<int64_t>(threadIdx.x) * kPerThread;
    if (base < n) {
      load4(xs + base, xv);
      load4(us + base, uv);
    }
    for (long long t = t0; t < t1; ++t) {
      const int64_t bnext = base + TILE;
      real xq[4], uq[4];
      const bool more = (t + 1 < t1) && bnext < n;
      if (more) {
        load4(xs + bnext, xq);
        load4(us + bnext, uq);
      }
      if (base < n) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (xv[q] > real(0) && xv[q] < Nr) {  // live (dead slots hold -1)
            const real Ef = gather<real>(Es2, xv[q]);
            const real un = fma(kap, Ef, uv[q]);
            const real xn = xv[q] + un;
            cfl = max(cfl, __float_as_uint(fabsf(static_cast<float>(un))));
            if (!(xn > real(0) && xn < Nr)) {  // absorbed (a non-finite value counts at x = d)
              const int el = (xn <= real(0)) ? 0 : 1;
              if (el) ++a1; else ++a0;
              if (s == CP_IONS) {
                const int slot = atomicAdd(&s_abs_n, 1);
                if (slot < abs_cap) {
                  AbsRecE r;
                  r.id = ids[base + q];
                  r.inst_el = static_cast<uint32_t>(2 * cur + el);
                  r.u = static_cast<double>(un);
                  my_abs[slot] = r;
                } else {
                  atomicCAS(&S->status, 0, CP_ERR_CAPACITY);
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
        fold_any(A, Bc, Gs, N, sign);
        __syncthreads();
        since = 0;
      }
    }
    __syncthreads();
    fold_any(A, Bc, Gs, N, sign);
    a0 = warp_sum_u(a0);
    a1 = warp_sum_u(a1);
    if (lane_id() == 0) {
      if (a0) atomicAdd(&s_cnt[0][s], static_cast<unsigned long long>(a0));
      if (a1) atomicAdd(&s_cnt[1][s], static_cast<unsigned long long>(a1));
    }
    u = t_end;
    __syncthreads();
    if (threadIdx.x == 0) s_j = j + 1;
    __syncthreads();
    // skip pairs with no tiles (stopped instances, empty species)
    if (threadIdx.x == 0) {
      int jj = s_j;
      while (jj < 3 * E && off[jj + 1] == off[jj] && off[jj] < u1) ++jj;
      s_j = jj;
    }
    __syncthreads();
  }
  if (cur >= 0) flush();

  // --- secondary emission from the ions this CTA saw absorbed ---------------
  const int na = min(s_abs_n, abs_cap);
  for (int r0 = 0; r0 < na; r0 += THREADS) {
    const int r = r0 + threadIdx.x;
    if (r >= na) break;
    const AbsRecE rec = my_abs[r];
    const int inst = static_cast<int>(rec.inst_el >> 1), el = static_cast<int>(rec.inst_el & 1u);
    const Bufs& B = Ball[inst];
    const DevParams* Pi = B.P;
    DevState* Si = B.S;
    const int64_t step = Si->level;
    const int Ni = Pi->N;
    const double dx = Pi->dx, dt = Pi->dt;
    const double v = __ddiv_rn(__dmul_rn(rec.u, dx), dt);
    const double Eev = __ddiv_rn(__dmul_rn(__dmul_rn(__dmul_rn(0.5, Pi->m_i), v), v), Pi->e);
    const int nse = see_count(Pi, Eev, rec.id, step);
    if (el == 0) {
      atomicAdd(reinterpret_cast<unsigned long long*>(&Si->ion_energy_q),
                static_cast<unsigned long long>(__double2ll_rn(Eev * 256.0)));
      if (nse) atomicAdd(reinterpret_cast<unsigned long long*>(&Si->conv_count),
                         static_cast<unsigned long long>(static_cast<long long>(nse)));
    }
    if (nse == 0) continue;
    atomicAdd(&Si->emitted[el], static_cast<unsigned long long>(nse));
    const unsigned long long wb =
        atomicAdd(reinterpret_cast<unsigned long long*>(&Si->n_alloc[CP_SECONDARIES]),
                  static_cast<unsigned long long>(nse));
    real* xs = reinterpret_cast<real*>(Si->xi[CP_SECONDARIES]);
    real* us = reinterpret_cast<real*>(Si->u[CP_SECONDARIES]);
    for (int jn = 0; jn < nse; ++jn) {
      double frac;
      const double vse = see_speed(Pi, rec.id, step, jn, &frac);
      const double use = vse * dt / dx;
      const double xd = (el == 0) ? __dmul_rn(use, frac) : __dsub_rn(static_cast<double>(Ni), __dmul_rn(use, frac));
      const real xr = nudge_inside<real>(xd, Ni);
      const real ur = static_cast<real>(el == 0 ? use : -use);
      const unsigned long long slot = wb + static_cast<unsigned long long>(jn);
      if (slot < static_cast<unsigned long long>(Pi->cap[CP_SECONDARIES])) {
        xs[slot] = xr;
        us[slot] = ur;
        deposit_global<real>(B.G, Ni, xr, -1LL);
      } else {
        atomicCAS(&Si->status, 0, CP_ERR_CAPACITY);
      }
    }
  }

  // --- beam ions of the instances this CTA serves (i = blockIdx.x mod grid) --
  for (int inst = blockIdx.x; inst < E; inst += gridDim.x) {
    const Bufs& B = Ball[inst];
    const DevParams* Pi = B.P;
    DevState* Si = B.S;
    const int Bn = Pi->beam_per_step;
    if (Bn <= 0 || ldcg(&Si->status) != 0) continue;
    const int64_t step = Si->level;
    const int Ni = Pi->N;
    const double dx = Pi->dx, dt = Pi->dt;
    real* xs = reinterpret_cast<real*>(Si->xi[CP_IONS]);
    real* us = reinterpret_cast<real*>(Si->u[CP_IONS]);
    uint32_t* ids = Si->id;
    const uint32_t id0 = Si->beam_id_base;
    for (int k0 = 0; k0 < Bn; k0 += THREADS) {
      const int k = k0 + threadIdx.x;
      const bool act = k < Bn;
      const unsigned ball = __ballot_sync(0xffffffffu, act);
      unsigned long long wbase = 0ULL;
      if (lane_id() == 0 && ball)
        wbase = atomicAdd(reinterpret_cast<unsigned long long*>(&Si->n_alloc[CP_IONS]),
                          static_cast<unsigned long long>(__popc(ball)));
      wbase = __shfl_sync(0xffffffffu, wbase, 0);
      if (act) {
        const U64x4 wv = philox4x64_10(static_cast<uint64_t>(k), static_cast<uint64_t>(step), 0, 0,
                                       Pi->seed, kTagBeam);
        const double frac = u01(wv.w[0]);
        double ub;
        if constexpr (sizeof(real) == 4) {  // the single FP32 gap's arithmetic
          ub = beam_speed_fp32(Pi, u01(wv.w[1]));
        } else {  // the single FP64 gap's: the definition's order of operations
          const double Eb = (Pi->beam_mode == 0)
                                ? Pi->beam_E_eV
                                : __dadd_rn(Pi->beam_Emin_eV, __dmul_rn(__dsub_rn(Pi->beam_Emax_eV, Pi->beam_Emin_eV), u01(wv.w[1])));
          const double v = sqrt(2.0 * Eb * Pi->e / Pi->m_i);
          ub = v * dt / dx;
        }
        const real xr = nudge_inside<real>(__dsub_rn(static_cast<double>(Ni), __dmul_rn(ub, frac)), Ni);
        const unsigned long long slot =
            wbase + static_cast<unsigned long long>(__popc(ball & ((1u << lane_id()) - 1u)));
        if (slot < static_cast<unsigned long long>(Pi->cap[CP_IONS])) {
          xs[slot] = xr;
          us[slot] = static_cast<real>(-ub);
          ids[slot] = id0 + static_cast<uint32_t>(step * Bn + k);
          deposit_global<real>(B.G, Ni, xr, 1LL);
        } else {
          atomicCAS(&Si->status, 0, CP_ERR_CAPACITY);
        }
      }
    }
    if (threadIdx.x == 0) atomicAdd(&Si->injected, static_cast<unsigned long long>(Bn));
  }
}

// ---------------------------------------------------------------------------
// Removal of absorbed particles over the flat (instance, species, tile) list
// ---------------------------------------------------------------------------
template <typename real>
__global__ void __launch_bounds__(kThreads) k_compact_ens(const Bufs* __restrict__ Ball, int E) {
  constexpr int TILE = kThreads * kPerThread;
  __shared__ int off[kEnsMaxEntries + 1];
  __shared__ int wsum[kThreads / 32];
  tile_offsets<kThreads>(Ball, E, TILE, off, wsum);
  const long long U = off[3 * E];
  // tiles are dealt round-robin: unit t -> its (instance, species) by search
  for (long long t = blockIdx.x; t < U; t += gridDim.x) {
    int lo = 0, hi = 3 * E;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (off[mid] <= t) lo = mid;
      else hi = mid;
    }
    const int inst = lo / 3, s = lo % 3;
    DevState* S = Ball[inst].S;
    const real* xs = reinterpret_cast<const real*>(S->xi[s]);
    const real* us = reinterpret_cast<const real*>(S->u[s]);
    real* xd = reinterpret_cast<real*>(S->xi_alt[s]);
    real* ud = reinterpret_cast<real*>(S->u_alt[s]);
    const uint32_t* is = S->id;
    uint32_t* id_d = S->id_alt;
    const int64_t n = S->n_proc[s];
    const int64_t base = (t - off[lo]) * TILE + static_cast<int64_t>(threadIdx.x) * kPerThread;
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

// One thread per instance: pad the packed stores to whole vectors and swap.
template <typename real>
__global__ void k_swap_ens(const Bufs* __restrict__ Ball, int E) {
  const int inst = blockIdx.x * blockDim.x + threadIdx.x;
  if (inst >= E) return;
  DevState* S = Ball[inst].S;
  if (S->status != 0) return;
  for (int s = 0; s < kSpecies; ++s) {
    const long long cnt = static_cast<long long>(S->compact_n[s]);
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
  uint32_t* t2 = S->id;
  S->id = S->id_alt;
  S->id_alt = t2;
}

// ---------------------------------------------------------------------------
// Host-side launchers
// ---------------------------------------------------------------------------
size_t push_ens_smem_bytes(int n_max, int precision, int E) {
  const size_t es = (precision == CP_FP32) ? 4 : 8;
  return align16(sizeof(long long) * (n_max + 1)) + align16(sizeof(unsigned int) * 2 * n_max) +
         align16(2 * es * (n_max + 1)) + align16(sizeof(int) * (3 * E + 1));
}

int ens_max_instances() { return kEnsMaxEntries / 3; }

template <typename real, int T>
static const void* push_ens_fn() {
  return reinterpret_cast<const void*>(k_push_ens<real, T>);
}

static const void* push_ens_kernel(int precision, int threads) {
  if (precision == CP_FP32) {
    if (threads == 256) return push_ens_fn<float, 256>();
    if (threads == 1024) return push_ens_fn<float, 1024>();
    return push_ens_fn<float, 512>();
  }
  if (threads == 256) return push_ens_fn<double, 256>();
  if (threads == 1024) return push_ens_fn<double, 1024>();
  return push_ens_fn<double, 512>();
}

// Resident CTAs per SM of the ensemble push for a block size (0: not launchable).
cudaError_t push_ens_occupancy(int precision, int threads, size_t smem, int* per_sm) {
  const void* fn = push_ens_kernel(precision, threads);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, threads, smem);
}

cudaError_t push_ens_launch(int precision, int threads, int grid, size_t smem, const Bufs* Ball,
                            int E, int n_max, void* abs, int abs_cap, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  AbsRecE* a = static_cast<AbsRecE*>(abs);
  if (precision == CP_FP32) {
    if (threads == 256) return cudaLaunchKernelEx(&cfg, k_push_ens<float, 256>, Ball, E, n_max, a, abs_cap);
    if (threads == 1024) return cudaLaunchKernelEx(&cfg, k_push_ens<float, 1024>, Ball, E, n_max, a, abs_cap);
    return cudaLaunchKernelEx(&cfg, k_push_ens<float, 512>, Ball, E, n_max, a, abs_cap);
  }
  if (threads == 256) return cudaLaunchKernelEx(&cfg, k_push_ens<double, 256>, Ball, E, n_max, a, abs_cap);
  if (threads == 1024) return cudaLaunchKernelEx(&cfg, k_push_ens<double, 1024>, Ball, E, n_max, a, abs_cap);
  return cudaLaunchKernelEx(&cfg, k_push_ens<double, 512>, Ball, E, n_max, a, abs_cap);
}

size_t abs_rec_ens_bytes() { return sizeof(AbsRecE); }

__global__ void k_status_ens(const Bufs* __restrict__ Ball, int E, int* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < E) out[i] = Ball[i].S->status;
}

cudaError_t status_ens_launch(const Bufs* Ball, int E, int* out, cudaStream_t st) {
  k_status_ens<<<(E + 127) / 128, 128, 0, st>>>(Ball, E, out);
  return cudaGetLastError();
}

cudaError_t compact_ens_launch(int precision, const Bufs* Ball, int E, int grid, cudaStream_t st) {
  if (precision == CP_FP32) {
    k_compact_ens<float><<<grid, kThreads, 0, st>>>(Ball, E);
    if (cudaGetLastError() != cudaSuccess) return cudaGetLastError();
    k_swap_ens<float><<<(E + 127) / 128, 128, 0, st>>>(Ball, E);
  } else {
    k_compact_ens<double><<<grid, kThreads, 0, st>>>(Ball, E);
    if (cudaGetLastError() != cudaSuccess) return cudaGetLastError();
    k_swap_ens<double><<<(E + 127) / 128, 128, 0, st>>>(Ball, E);
  }
  return cudaGetLastError();
}

}  // namespace cpk
