// cp_noalloc.cu -- an allocation-free variant of the ion push.
//
// Some callers cannot call cudaMalloc: a simulation step embedded in a
// real-time control loop or a host process that must not grow device
// memory after start-up, or code that runs while another component owns the
// allocator.  For them cp_push_ions_noalloc pushes one FP32 ion population
// through one step (gather, kick, drift, absorption, ion-induced secondary
// emission, deposit) using only buffers the caller passes in.  The scratch
// it needs -- the list of ions absorbed in the push, which the context path
// keeps in memory it allocates -- lives in the file-scope array below, which
// every GPU that loads this library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "cp_device.cuh"

namespace cpk_na {

using cpk::AbsRec;
using cpk::kTagSee;
using cpk::philox4x64_10;
using cpk::u01;
using cpk::U64x4;

constexpr int kThreads = 256;
constexpr int kMaxCells = 4096;          // shared-memory grid limit
constexpr int64_t kMaxIons = 1 << 19;    // absorbed-ion records the scratch can hold
constexpr int kCounters = 16;            // [0] list length, [1] SE count, [2] overflow, tallies

// Scratch: counters, then one record per ion that may be absorbed (8 MiB + 128 B).
struct Scratch {
  unsigned long long counters[kCounters];
  AbsRec rec[kMaxIons];
};
static __device__ __align__(256) Scratch g_scratch;

// Tally slots in Scratch::counters
enum { kListLen = 0, kSeCount = 1, kOverflow = 2, kAbs0 = 3, kAbs1 = 4, kEmit0 = 5, kEmit1 = 6, kConv = 7,
       kStatus = kCounters - 1 };

struct Params {
  int N;
  float kap;         // kick factor (half or full) in cells/step^2 per V/m
  double dx, dt, m_i, e, m_e;
  double see_scale, gamma_coef, gamma_max, E_ref_eV, see_vth;
  uint64_t seed;
  int64_t step;
};

__device__ __forceinline__ unsigned lane() { return threadIdx.x & 31u; }

__device__ __forceinline__ void dep_atomic(long long* G, int N, float x, long long sign) {
  const float fl = floorf(x);
  const int i = static_cast<int>(fl);
  const long long w1 = static_cast<long long>(__float2uint_rz((x - fl) * 65536.0f));
  long long w0 = 65536LL - w1, w1b = w1;
  if (i == 0) w0 <<= 1;
  if (i == N - 1) w1b <<= 1;
  atomicAdd(reinterpret_cast<unsigned long long*>(&G[i]), static_cast<unsigned long long>(sign * w0));
  atomicAdd(reinterpret_cast<unsigned long long*>(&G[i + 1]), static_cast<unsigned long long>(sign * w1b));
}

// Push, absorb (absorbed ions compacted into the scratch list with
// warp-ballot appends) and deposit of the survivors into the caller's grid.
__global__ void __launch_bounds__(kThreads) k_push_ions(Params p, Scratch* sc, const double* E,
                                                        float* xi, float* u, const uint32_t* id,
                                                        int64_t n, long long* G) {
  extern __shared__ __align__(16) unsigned char smem_na[];
  const int N = p.N;
  long long* Gs = reinterpret_cast<long long*>(smem_na);        // N + 1
  float2* tab = reinterpret_cast<float2*>(Gs + (N + 1));         // N + 1
  // gather table: pair k = (Ep_k, Ep_{k+1} - Ep_k), ends repeated
  for (int k = threadIdx.x; k <= N; k += kThreads) {
    const float e0 = static_cast<float>(E[k == 0 ? 0 : k - 1]);
    const float e1 = (k >= 1 && k < N) ? static_cast<float>(E[k]) : e0;
    tab[k] = make_float2(e0, e1 - e0);
    Gs[k] = 0;
  }
  __syncthreads();
  const float Nr = static_cast<float>(N);
  unsigned long long a0 = 0, a1 = 0;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * kThreads;
  const int64_t trips = (n + stride - 1) / stride;  // uniform: warps stay converged
  for (int64_t t = 0; t < trips; ++t) {
    const int64_t k = t * stride + static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x;
    bool absorbed = false;
    int el = 0;
    float un = 0.f;
    if (k < n) {
      const float x = xi[k];
      if (x > 0.f && x < Nr) {
        const float s = x - 0.5f;
        const float jf = floorf(s);
        const float2 e = tab[static_cast<int>(jf) + 1];
        un = fmaf(p.kap, fmaf(s - jf, e.y, e.x), u[k]);
        const float xn = x + un;
        if (!(xn > 0.f && xn < Nr)) {
          absorbed = true;
          el = (xn <= 0.f) ? 0 : 1;
          xi[k] = -1.f;
          u[k] = 0.f;
        } else {
          xi[k] = xn;
          u[k] = un;
          const float fl = floorf(xn);
          const int i = static_cast<int>(fl);
          const long long w1 = static_cast<long long>(__float2uint_rz((xn - fl) * 65536.0f));
          long long w0 = 65536LL - w1, w1b = w1;
          if (i == 0) w0 <<= 1;
          if (i == N - 1) w1b <<= 1;
          atomicAdd(reinterpret_cast<unsigned long long*>(&Gs[i]), static_cast<unsigned long long>(w0));
          atomicAdd(reinterpret_cast<unsigned long long*>(&Gs[i + 1]), static_cast<unsigned long long>(w1b));
        }
      }
    }
    // warp-ballot compaction of the absorbed ions into the scratch list
    const unsigned ball = __ballot_sync(0xffffffffu, absorbed);
    unsigned long long base = 0;
    if (lane() == 0 && ball)
      base = atomicAdd(&sc->counters[kListLen], static_cast<unsigned long long>(__popc(ball)));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (absorbed) {
      const unsigned long long slot = base + __popc(ball & ((1u << lane()) - 1u));
      AbsRec r;
      r.id = id[k];
      r.electrode = static_cast<uint32_t>(el);
      r.u = static_cast<double>(un);
      sc->rec[slot] = r;  // slot < n <= kMaxIons: every ion fits
      if (el) ++a1; else ++a0;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k <= N; k += kThreads)
    if (Gs[k]) atomicAdd(reinterpret_cast<unsigned long long*>(&G[k]), static_cast<unsigned long long>(Gs[k]));
  if (a0) atomicAdd(&sc->counters[kAbs0], a0);
  if (a1) atomicAdd(&sc->counters[kAbs1], a1);
}

// Secondary emission from the listed impacts (same arithmetic and draws as
// the context path); electrons appended to the caller's arrays.
__global__ void __launch_bounds__(kThreads) k_see(Params p, Scratch* sc, float* se_xi, float* se_u,
                                                  int64_t se_cap, long long* G) {
  const unsigned long long len = sc->counters[kListLen];
  const int64_t stride = static_cast<int64_t>(gridDim.x) * kThreads;
  const int64_t trips = (static_cast<int64_t>(len) + stride - 1) / stride;
  const int N = p.N;
  const double pi = 3.14159265358979323846;
  for (int64_t t = 0; t < trips; ++t) {
    const int64_t r = t * stride + static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x;
    const bool act = r < static_cast<int64_t>(len);
    int nse = 0;
    AbsRec rec;
    rec.id = 0; rec.electrode = 0; rec.u = 0.0;
    double Eev = 0.0;
    if (act) {
      rec = sc->rec[r];
      const double v = __ddiv_rn(__dmul_rn(rec.u, p.dx), p.dt);
      Eev = __ddiv_rn(__dmul_rn(__dmul_rn(__dmul_rn(0.5, p.m_i), v), v), p.e);
      double g = __dmul_rn(__dmul_rn(p.see_scale, p.gamma_coef), __dsqrt_rn(__ddiv_rn(Eev, p.E_ref_eV)));
      if (g > p.gamma_max) g = p.gamma_max;
      if (!(g > 0.0)) g = 0.0;
      const U64x4 w = philox4x64_10(rec.id, static_cast<uint64_t>(p.step), 0, 0, p.seed, kTagSee);
      const double fl = floor(g);
      nse = static_cast<int>(fl) + ((u01(w.w[0]) < __dsub_rn(g, fl)) ? 1 : 0);
      if (nse) atomicAdd(&sc->counters[rec.electrode ? kEmit1 : kEmit0], static_cast<unsigned long long>(nse));
      if (rec.electrode == 0 && nse)
        atomicAdd(&sc->counters[kConv], static_cast<unsigned long long>(nse));
    }
    int incl = nse;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (static_cast<int>(lane()) >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long base = 0;
    if (lane() == 31 && total)
      base = atomicAdd(&sc->counters[kSeCount], static_cast<unsigned long long>(total));
    base = __shfl_sync(0xffffffffu, base, 31);
    for (int j = 0; j < nse; ++j) {
      const U64x4 wv = philox4x64_10(rec.id, static_cast<uint64_t>(p.step), static_cast<uint64_t>(1 + j), 0,
                                     p.seed, kTagSee);
      const double ua = u01(wv.w[0]), ub = u01(wv.w[1]), frac = u01(wv.w[2]);
      const double z = sqrt(-2.0 * log(ua)) * cos(2.0 * pi * ub);
      const double use = p.see_vth * fabs(z) * p.dt / p.dx;
      const double xd = (rec.electrode == 0) ? __dmul_rn(use, frac) : __dsub_rn(static_cast<double>(N), __dmul_rn(use, frac));
      float xr = static_cast<float>(xd);
      if (xr >= static_cast<float>(N)) xr = nextafterf(static_cast<float>(N), 0.f);
      if (xr <= 0.f) xr = 1.17549435e-38f;
      const unsigned long long slot = base + static_cast<unsigned long long>(incl - nse + j);
      if (slot < static_cast<unsigned long long>(se_cap)) {
        se_xi[slot] = xr;
        se_u[slot] = static_cast<float>(rec.electrode == 0 ? use : -use);
        dep_atomic(G, N, xr, -1LL);
      } else {
        sc->counters[kOverflow] = 1ULL;
      }
    }
  }
}

// The call's six counts written on the device (no host round trip): [0]
// absorbed at x = 0, [1] absorbed at x = d, [2] emitted at x = 0, [3] emitted
// at x = d, [4] electrons written (at most se_cap), [5] convection count at
// x = 0.  status[0] = 1 when emitted electrons did not fit in se_cap.
__global__ void k_counts(const Scratch* sc, int64_t se_cap, int64_t* counts, unsigned long long* status) {
  const unsigned long long se = sc->counters[kSeCount];
  const unsigned long long cap = static_cast<unsigned long long>(se_cap);
  counts[0] = static_cast<int64_t>(sc->counters[kAbs0]);
  counts[1] = static_cast<int64_t>(sc->counters[kAbs1]);
  counts[2] = static_cast<int64_t>(sc->counters[kEmit0]);
  counts[3] = static_cast<int64_t>(sc->counters[kEmit1]);
  counts[4] = static_cast<int64_t>(se < cap ? se : cap);
  counts[5] = static_cast<int64_t>(sc->counters[kAbs0]) + static_cast<int64_t>(sc->counters[kEmit0]);
  status[0] = (sc->counters[kOverflow] || se > cap) ? 1ULL : 0ULL;
}

// Device address of the scratch array (and the push kernel's shared-memory
// limit), set up once per device with that device current.
std::mutex g_mu;
Scratch* g_addr[64] = {};

int scratch_address(int dev, Scratch** out) {
  if (dev < 0 || dev >= 64) return CP_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return CP_ERR_CUDA;
    }
    if (cudaFuncSetAttribute(k_push_ions, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(16 * (kMaxCells + 1))) != cudaSuccess) {
      cudaGetLastError();
      return CP_ERR_CUDA;
    }
    g_addr[dev] = static_cast<Scratch*>(ptr);
  }
  *out = g_addr[dev];
  return CP_OK;
}

}  // namespace cpk_na

extern "C" int cp_push_ions_noalloc(const cp_gap* gap, const cp_see_beam* see, double dt, uint64_t seed,
                                    int64_t step, int32_t half_kick, const double* E, float* xi,
                                    float* u, const uint32_t* id, int64_t n, int64_t* G, float* se_xi,
                                    float* se_u, int64_t se_cap, int64_t* counts, void* stream) {
  using namespace cpk_na;
  if (!gap || !see || !E || !G || !counts || n < 0 || (n > 0 && (!xi || !u || !id)) || se_cap < 0 ||
      (se_cap > 0 && (!se_xi || !se_u)) || !(dt > 0) || !(gap->d > 0) || !(gap->m_i > 0) ||
      !(gap->e > 0) || !(gap->m_e > 0) || step < 0)
    return CP_ERR_ARG;
  // the SEE law as cp_create accepts it: a bounded mean yield keeps the
  // per-impact draw loop and the warp scan of counts small, and a finite,
  // non-negative emission temperature keeps the emitted positions finite
  if (!(see->gamma_max >= 0.0 && see->gamma_max <= 14.0) || !(see->scale >= 0.0) ||
      !std::isfinite(see->scale) || !(see->gamma_coef >= 0.0) || !std::isfinite(see->gamma_coef) ||
      !(see->T_emit_eV >= 0.0) || !std::isfinite(see->T_emit_eV) || !(see->E_ref_eV >= 0.0) ||
      !std::isfinite(see->E_ref_eV) || see->count_law != CP_SEE_COUNT_BERNOULLI ||
      see->energy_law != CP_SEE_ENERGY_MAXWELL)
    return CP_ERR_ARG;
  if (gap->n_cells < 2 || gap->n_cells > kMaxCells) return CP_ERR_ARG;  // shared-memory grid limit
  if (n > kMaxIons) return CP_ERR_CAPACITY;  // beyond the scratch array: every ion might be absorbed
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CP_ERR_CUDA;
  Scratch* sc = nullptr;
  const int rc = scratch_address(dev, &sc);
  if (rc != CP_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int N = gap->n_cells;
  Params p;
  p.N = N;
  p.dx = gap->d / N;
  p.dt = dt;
  p.m_i = gap->m_i;
  p.e = gap->e;
  p.m_e = gap->m_e;
  const double kappa = gap->e * dt * dt / (gap->m_i * p.dx);
  p.kap = static_cast<float>(half_kick ? 0.5 * kappa : kappa);
  p.see_scale = see->scale;
  p.gamma_coef = see->gamma_coef;
  p.gamma_max = see->gamma_max;
  p.E_ref_eV = see->E_ref_eV > 0 ? see->E_ref_eV : 1000.0;
  p.see_vth = std::sqrt(gap->e * see->T_emit_eV / gap->m_e);
  p.seed = seed;
  p.step = step;
  // the scratch keeps the previous call's contents: its counters start at zero
  if (cudaMemsetAsync(sc->counters, 0, sizeof(sc->counters), st) != cudaSuccess ||
      cudaMemsetAsync(G, 0, sizeof(int64_t) * (N + 1), st) != cudaSuccess)
    return CP_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CP_ERR_CUDA;
  const int grid = 2 * sms;
  long long* Gl = reinterpret_cast<long long*>(G);
  k_push_ions<<<grid, kThreads, 16 * (N + 1), st>>>(p, sc, E, xi, u, id, n, Gl);
  k_see<<<grid, kThreads, 0, st>>>(p, sc, se_xi, se_u, se_cap, Gl);
  // counts on the device; one copy of the overflow flag back for the status
  unsigned long long* flag = &sc->counters[kStatus];
  k_counts<<<1, 1, 0, st>>>(sc, se_cap, counts, flag);
  if (cudaGetLastError() != cudaSuccess) return CP_ERR_CUDA;
  unsigned long long overflow = 0;
  if (cudaMemcpyAsync(&overflow, flag, sizeof(overflow), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return CP_ERR_CUDA;
  if (overflow) return CP_ERR_CAPACITY;
  return CP_OK;
}
