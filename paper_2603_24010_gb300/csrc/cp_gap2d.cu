// cp_gap2d.cu -- the 2D planar gap: x normal to the electrodes, y periodic.
//
// The cycle of the 1D gap (arXiv 2603.24010) in two dimensions, arranged for
// the GB300:
//
// * Particle store: structure of arrays per species (x, u in the 1D state's
//   buffers, y, w here), kept sorted by 32 x 32-cell tiles (counting sort
//   every `sort_every` steps, which also drops absorbed particles); each
//   tile's segment starts on a 16-byte boundary.
// * k2_push: a persistent grid takes work items of up to 32768 particles of
//   one tile from an atomic queue; the item's field window (the tile plus 4
//   cells of halo, E_x and E_y, each node paired with its neighbour in y)
//   is staged in shared memory, and its charge goes into five exact 32-bit
//   sums per cell (count, sum of wx1, sum of wy1, high and low parts of the
//   sum of wx1 wy1), from which the flush forms every node's int64 charge.
//   Particles that left their window since the sort (and the unsorted tail
//   of emitted electrons and beam ions) gather from and deposit into global
//   memory directly, with the same arithmetic.
// * Solve: each row of the grid is summed exactly (the int64 column sums are
//   the 1D coupled problem of Sec. 2.4.2/2.4.3, solved by the 1D cluster
//   solve, circuit and history included) and Fourier-transformed in y
//   (radix-2 FFT in shared memory, FP32); every transverse mode k != 0
//   solves its tridiagonal system in x with phi = 0 on both electrodes
//   (Thomas, one thread per mode); the inverse transform and the 1D field
//   give E_x = E_0(x) + dE_x and E_y on the staggered grid.
#include <cuda_runtime.h>

#include <algorithm>

#include "cp_common.cuh"
#include "cp_gap2d.cuh"

namespace cpk {

// ---------------------------------------------------------------------------
// Gather and deposit helpers (global coordinates; the window only changes
// where the values are read from or added to)
// ---------------------------------------------------------------------------
struct Stencil2 {
  int i, i1, j, j1;   // E_x: x half-grid indices, y node indices
  float t, v;
  int a, a1, jj, jj1; // E_y: x node indices, y half-grid indices
  float fx, vy;
};

__device__ __forceinline__ int wrapi(int j, int N) { return j < 0 ? j + N : (j >= N ? j - N : j); }
__device__ __forceinline__ int modp(int j, int N) { const int r = j % N; return r < 0 ? r + N : r; }

__device__ __forceinline__ Stencil2 stencil2(const Dev2D& D, float x, float y) {
  Stencil2 st;
  const float s = x - 0.5f;
  float sf = floorf(s);
  int i = static_cast<int>(sf);
  float t = s - sf;
  if (s < 0.0f) {
    i = 0;
    t = 0.0f;
  } else if (i >= D.Nx - 1) {
    i = D.Nx - 1;
    t = 0.0f;
  }
  st.i = i;
  st.i1 = min(i + 1, D.Nx - 1);
  st.t = t;
  const float yf = floorf(y);
  st.j = wrapi(static_cast<int>(yf), D.Ny);
  st.j1 = wrapi(st.j + 1, D.Ny);
  st.v = y - yf;
  const float xf = floorf(x);
  st.a = static_cast<int>(xf);
  st.a1 = st.a + 1;
  st.fx = x - xf;
  const float sy = y - 0.5f;
  const float syf = floorf(sy);
  st.jj = wrapi(static_cast<int>(syf), D.Ny);
  st.jj1 = wrapi(st.jj + 1, D.Ny);
  st.vy = sy - syf;
  return st;
}

__device__ __forceinline__ float bilin(float f00, float f10, float f01, float f11, float a, float b) {
  return (1.0f - b) * ((1.0f - a) * f00 + a * f10) + b * ((1.0f - a) * f01 + a * f11);
}

// window index of a 2x2 stencil's origin node (gx, gy) when the whole
// stencil lies in the window (origin at most kW2-2 from the window's edge);
// -1 otherwise
__device__ __forceinline__ int win_rel(int gx, int gy, int ox, int oy, int Ny) {
  const int lx = gx - ox;
  int ly = gy - oy;
  if (ly < 0) ly += Ny;
  else if (ly >= Ny) ly -= Ny;
  if (static_cast<unsigned>(lx) > static_cast<unsigned>(kW2 - 2) ||
      static_cast<unsigned>(ly) > static_cast<unsigned>(kW2 - 2))
    return -1;
  return lx * kW2 + ly;
}

// window coordinates of a global node (x index gx, y index gy); -1 if outside
__device__ __forceinline__ int win_index(int gx, int gy, int ox, int oy, int Ny) {
  const int lx = gx - ox;
  int ly = gy - oy;
  if (ly < 0) ly += Ny;
  if (ly >= Ny) ly -= Ny;
  if (lx < 0 || lx >= kW2 || ly < 0 || ly >= kW2) return -1;
  return lx * kW2 + ly;
}

// fixed-point bilinear weights floor(frac 2^16) per axis: the corner
// products sum to 2^32 per macroparticle (x - floor(x) and the power-of-two
// scaling are exact, so the truncation decides alone)
__device__ __forceinline__ void deposit_weights(float x, float y, int Ny, int* i, int* j, int* j1,
                                                unsigned long long* w00, unsigned long long* w10,
                                                unsigned long long* w01, unsigned long long* w11) {
  const float xf = floorf(x), yf = floorf(y);
  *i = static_cast<int>(xf);
  *j = static_cast<int>(yf);
  *j1 = wrapi(*j + 1, Ny);
  const unsigned int wx1 = __float2uint_rz((x - xf) * 65536.0f);
  const unsigned int wy1 = __float2uint_rz((y - yf) * 65536.0f);
  const unsigned int wx0 = 65536u - wx1, wy0 = 65536u - wy1;
  *w00 = static_cast<unsigned long long>(wx0) * wy0;
  *w10 = static_cast<unsigned long long>(wx1) * wy0;
  *w01 = static_cast<unsigned long long>(wx0) * wy1;
  *w11 = static_cast<unsigned long long>(wx1) * wy1;
}

// cell (i, j) of a particle and its per-axis weights wx1 = floor(frac(x) 2^16),
// wy1 = floor(frac(y) 2^16), as deposit_weights forms them
__device__ __forceinline__ void cell_weights(float x, float y, int* i, int* j, unsigned int* wx1,
                                             unsigned int* wy1) {
  const float xf = floorf(x), yf = floorf(y);
  *i = static_cast<int>(xf);
  *j = static_cast<int>(yf);
  *wx1 = __float2uint_rz((x - xf) * 65536.0f);
  *wy1 = __float2uint_rz((y - yf) * 65536.0f);
}

__device__ __forceinline__ void atomic_add_i64(long long* p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(v));
}

__device__ __forceinline__ void deposit2_global(const Dev2D& D, float x, float y, long long sign) {
  int i, j, j1;
  unsigned long long w00, w10, w01, w11;
  deposit_weights(x, y, D.Ny, &i, &j, &j1, &w00, &w10, &w01, &w11);
  const long long di = (i == 0) ? 2 : 1, di1 = (i + 1 == D.Nx) ? 2 : 1;
  long long* G = D.G2;
  const long long r0 = static_cast<long long>(i) * D.Ny, r1 = static_cast<long long>(i + 1) * D.Ny;
  if (w00) atomic_add_i64(&G[r0 + j], sign * di * static_cast<long long>(w00));
  if (w10) atomic_add_i64(&G[r1 + j], sign * di1 * static_cast<long long>(w10));
  if (w01) atomic_add_i64(&G[r0 + j1], sign * di * static_cast<long long>(w01));
  if (w11) atomic_add_i64(&G[r1 + j1], sign * di1 * static_cast<long long>(w11));
}

// ---------------------------------------------------------------------------
// k2_push
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads2, 2)
k2_push(const DevParams* __restrict__ P, DevState* S, const Dev2D* __restrict__ Dp,
        const __grid_constant__ Dev2D Dc, int* __restrict__ item_ctr, AbsRec2* __restrict__ abs_all,
        int abs_cap) {
  // field window: each node holds its value and that of the next node in y
  // (one 8-byte load per stencil column)
  __shared__ float2 Exw[kW2 * kW2];
  __shared__ float2 Eyw[kW2 * kW2];
  // Deposit window, by cell (indexed like its lower corner node): the
  // particle count n, the sums sx, sy of the per-axis weights wx1, wy1 and
  // the high bits and low 16 bits of the sum sxy of wx1 wy1 (< 2^32 each).
  // The four corner weights of a particle are linear in these (A = 2^16):
  // w00 = A^2 - A wx1 - A wy1 + wx1 wy1, w10 = A wx1 - wx1 wy1,
  // w01 = A wy1 - wx1 wy1, w11 = wx1 wy1; the flush forms each node's exact
  // int64 sum from its four cells.  An item of at most 32768 particles keeps
  // every 32-bit sum below 2^31.
  extern __shared__ unsigned int cwin[];
  unsigned int* Cn = cwin;
  unsigned int* Cx = cwin + kW2 * kW2;
  unsigned int* Cy = cwin + 2 * kW2 * kW2;
  unsigned int* Ch = cwin + 3 * kW2 * kW2;
  unsigned int* Cl = cwin + 4 * kW2 * kW2;
  __shared__ int s_items[2 * kSpecies + 1];  // item offsets: sorted / tail per species
  __shared__ int s_abs_n, s_stop, s_over;
  __shared__ unsigned long long s_cnt[2][kSpecies];
  __shared__ unsigned long long s_emit[2];
  __shared__ long long s_conv, s_energy;
  __shared__ unsigned int s_cfl;

  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();
  // the fields fixed at creation come from the launch parameters; the sort
  // swaps the y, w buffers and sets n_sorted on the device, so those are read
  // from the device copy
  const Dev2D& D = Dc;
  if (threadIdx.x == 0) {
    s_stop = (ldcg(&S->status) != 0);
    s_abs_n = 0;
    s_over = 0;
    s_conv = 0;
    s_energy = 0;
    s_cfl = 0u;
    s_emit[0] = s_emit[1] = 0ULL;
    int acc = 0;
    for (int s = 0; s < kSpecies; ++s) {
      s_items[2 * s] = acc;
      acc += D.wi_off[s * (D.T + 1) + D.T];
      s_items[2 * s + 1] = acc;
      const long long tail = S->n_proc[s] - Dp->n_sorted[s];
      acc += static_cast<int>((tail + kChunk2 - 1) / kChunk2);
    }
    s_items[2 * kSpecies] = acc;
  }
  if (threadIdx.x < 2 * kSpecies) s_cnt[threadIdx.x / kSpecies][threadIdx.x % kSpecies] = 0ULL;
  __syncthreads();
  if (s_stop) return;
  const bool half = (S->pushed == 0);
  const int64_t step = S->level;
  const int Ny = D.Ny;
  AbsRec2* my_abs = abs_all + static_cast<size_t>(blockIdx.x) * abs_cap;
  unsigned int cfl = 0u;
  unsigned int a_cnt[2][kSpecies] = {{0u, 0u, 0u}, {0u, 0u, 0u}};

  const int n_items = s_items[2 * kSpecies];
  // Work items are taken from a queue (one atomic ticket per item): items
  // differ in size (whole and partial tiles, the unsorted tails), and a
  // fixed round-robin deal left CTAs idle while others finished theirs.
  // The last CTA out resets the queue for the next launch.
  __shared__ int s_item;
  for (;;) {
    __syncthreads();  // every thread has read the previous ticket
    if (threadIdx.x == 0) s_item = atomicAdd(&item_ctr[0], 1);
    __syncthreads();
    const int item = s_item;
    if (item >= n_items) break;
    int s = 0;
    while (item >= s_items[2 * s + 2]) ++s;
    const bool tail = item >= s_items[2 * s + 1];
    long long p0, p1;
    int ox = 0, oy = 0;
    bool win = false;
    if (!tail) {
      const int k = item - s_items[2 * s];
      const int* wo = D.wi_off + s * (D.T + 1);
      int lo = 0, hi = D.T;  // tile with wo[t] <= k < wo[t+1]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (wo[mid] <= k) lo = mid;
        else hi = mid;
      }
      const int t = lo;
      const int* ts = D.tile_start + s * (D.T + 1);
      p0 = ts[t] + static_cast<long long>(k - wo[t]) * kChunk2;
      p1 = min(static_cast<long long>(ts[t + 1]), p0 + kChunk2);
      ox = (t / D.nty) * kT2 - kH2 - 1;
      oy = (t % D.nty) * kT2 - kH2 - 1;
      win = D.use_win != 0;
      // stage the field window; zero the deposit window
      for (int q = threadIdx.x; win && q < kW2 * kW2; q += kThreads2) {
        const int lx = q / kW2, ly = q % kW2;
        const int gx = ox + lx;
        const int gy = wrapi(oy + ly, Ny);  // one wrap: Ny >= the window edge
        const int gy1 = wrapi(gy + 1, Ny);
        const long long r = static_cast<long long>(gx) * Ny;
        Exw[q] = (gx >= 0 && gx < D.Nx) ? make_float2(D.Ex[r + gy], D.Ex[r + gy1]) : make_float2(0.0f, 0.0f);
        Eyw[q] = (gx >= 0 && gx <= D.Nx) ? make_float2(D.Ey[r + gy], D.Ey[r + gy1]) : make_float2(0.0f, 0.0f);
        Cn[q] = Cx[q] = Cy[q] = Ch[q] = Cl[q] = 0u;
      }
      __syncthreads();
    } else {
      const int k = item - s_items[2 * s + 1];
      p0 = Dp->n_sorted[s] + static_cast<long long>(k) * kChunk2;
      p1 = min(static_cast<long long>(S->n_proc[s]), p0 + kChunk2);
    }
    float* xs = reinterpret_cast<float*>(S->xi[s]);
    float* us = reinterpret_cast<float*>(S->u[s]);
    float* ys = reinterpret_cast<float*>(Dp->y[s]);
    float* ws = reinterpret_cast<float*>(Dp->w[s]);
    const uint32_t* ids = S->id;
    const float kx = D.kx[half ? 0 : 1][s], ky = D.ky[half ? 0 : 1][s];
    const long long sign = (s == CP_IONS) ? 1LL : -1LL;
    for (long long b0 = p0; b0 < p1; b0 += kThreads2 * 4) {
      const long long base = b0 + static_cast<long long>(threadIdx.x) * 4;
      if (base < p1) {
        float xv[4], uv[4], yv[4], wv[4];
        load4(xs + base, xv);
        load4(us + base, uv);
        load4(ys + base, yv);
        load4(ws + base, wv);
        // Fast path, without divergent branches: a live particle whose
        // stencils lie in the window, that stays inside the gap and whose
        // deposit lands in the window (the common case).  Every other live
        // particle is flagged and takes the general path below, on its
        // unchanged values, with the same arithmetic.
        unsigned int slow = 0u;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float x = xv[q];
          const bool alive = (x > 0.0f && x < D.Nxf);
          const float xa = alive ? x : 1.0f, ya = alive ? yv[q] : 0.0f;  // defined indices for dead slots
          const Stencil2 st = stencil2(D, xa, ya);
          const int le = win_rel(st.i, st.j, ox, oy, Ny), lf = win_rel(st.a, st.jj, ox, oy, Ny);
          const bool gw = win && alive && le >= 0 && lf >= 0;
          const int e00 = gw ? le : 0, e10 = gw ? le + (st.i1 - st.i) * kW2 : 0;
          const int f00 = gw ? lf : 0, f10 = f00 + kW2;
          const float2 cx0 = Exw[e00], cx1 = Exw[e10], cy0 = Eyw[f00], cy1 = Eyw[f10];
          const float ex = bilin(cx0.x, cx1.x, cx0.y, cx1.y, st.t, st.v);
          const float ey = bilin(cy0.x, cy1.x, cy0.y, cy1.y, st.fx, st.vy);
          const float un = fmaf(kx, ex, uv[q]);
          const float wn = fmaf(ky, ey, wv[q]);
          const float xn = x + un;
          float yn = yv[q] + wn;
          if (yn < 0.0f) yn += D.Nyf;
          if (yn >= D.Nyf) yn -= D.Nyf;
          const bool inside = (xn > 0.0f && xn < D.Nxf) && (yn >= 0.0f && yn < D.Nyf);
          int i, j;
          unsigned int wx1, wy1;
          cell_weights(inside ? xn : 1.0f, inside ? yn : 0.0f, &i, &j, &wx1, &wy1);
          const int d00 = win ? win_rel(i, j, ox, oy, Ny) : -1;
          const bool good = gw && inside && d00 >= 0;
          if (good) {
            const unsigned int xy = wx1 * wy1;  // < 2^32
            atomicAdd(&Cn[d00], 1u);
            if (wx1) atomicAdd(&Cx[d00], wx1);
            if (wy1) atomicAdd(&Cy[d00], wy1);
            if (xy >> 16) atomicAdd(&Ch[d00], xy >> 16);
            if (xy & 0xFFFFu) atomicAdd(&Cl[d00], xy & 0xFFFFu);
            cfl = max(cfl, __float_as_uint(fmaxf(fabsf(un), fabsf(wn))));
            xv[q] = xn;
            uv[q] = un;
            yv[q] = yn;
            wv[q] = wn;
          } else if (alive) {
            slow |= 1u << q;
          }
        }
        if (slow) {  // the general path
  #pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (!((slow >> q) & 1u)) continue;
            const float x = xv[q];
            const Stencil2 st = stencil2(D, x, yv[q]);
            float ex, ey;
            // window origins of the two 2x2 stencils (the window is contiguous in
            // y, so the corners sit at +1 row / +1 column of their origin)
            const int le = win_rel(st.i, st.j, ox, oy, Ny), lf = win_rel(st.a, st.jj, ox, oy, Ny);
            if (win && le >= 0 && lf >= 0) {
              const int e00 = le, e10 = le + (st.i1 - st.i) * kW2;
              const int f00 = lf, f10 = lf + kW2;
              const float2 cx0 = Exw[e00], cx1 = Exw[e10], cy0 = Eyw[f00], cy1 = Eyw[f10];
              ex = bilin(cx0.x, cx1.x, cx0.y, cx1.y, st.t, st.v);
              ey = bilin(cy0.x, cy1.x, cy0.y, cy1.y, st.fx, st.vy);
            } else {
              const float* Ex = D.Ex;
              const float* Ey = D.Ey;
              const long long ri = static_cast<long long>(st.i) * Ny, ri1 = static_cast<long long>(st.i1) * Ny;
              const long long ra = static_cast<long long>(st.a) * Ny, ra1 = static_cast<long long>(st.a1) * Ny;
              ex = bilin(__ldg(&Ex[ri + st.j]), __ldg(&Ex[ri1 + st.j]), __ldg(&Ex[ri + st.j1]),
                         __ldg(&Ex[ri1 + st.j1]), st.t, st.v);
              ey = bilin(__ldg(&Ey[ra + st.jj]), __ldg(&Ey[ra1 + st.jj]), __ldg(&Ey[ra + st.jj1]),
                         __ldg(&Ey[ra1 + st.jj1]), st.fx, st.vy);
            }
            const float un = fmaf(kx, ex, uv[q]);
            const float wn = fmaf(ky, ey, wv[q]);
            const float xn = x + un;
            float yn = yv[q] + wn;
            if (yn < 0.0f) yn += D.Nyf;
            if (yn >= D.Nyf) yn -= D.Nyf;
            if (!(yn >= 0.0f && yn < D.Nyf)) {  // more than one period in a step (or not finite)
              yn -= D.Nyf * floorf(yn / D.Nyf);
              if (!(yn >= 0.0f && yn < D.Nyf)) yn = 0.0f;
            }
            cfl = max(cfl, __float_as_uint(fmaxf(fabsf(un), fabsf(wn))));
            if (!(xn > 0.0f && xn < D.Nxf)) {  // absorbed
              const int el = (xn <= 0.0f) ? 0 : 1;
              ++a_cnt[el][s];
              if (s == CP_IONS) {
                const int slot = atomicAdd(&s_abs_n, 1);
                if (slot < abs_cap) {
                  AbsRec2 r;
                  r.id = ids[base + q];
                  r.el = static_cast<uint32_t>(el);
                  r.u = un;
                  r.w = wn;
                  r.eta = yn;
                  r.pad = 0.0f;
                  my_abs[slot] = r;
                } else {
                  s_over = 1;
                }
              }
              xv[q] = -1.0f;
              uv[q] = 0.0f;
              yv[q] = 0.0f;
              wv[q] = 0.0f;
              continue;
            }
            xv[q] = xn;
            uv[q] = un;
            yv[q] = yn;
            wv[q] = wn;
            int i, j;
            unsigned int wx1, wy1;
            cell_weights(xn, yn, &i, &j, &wx1, &wy1);
            const int d00 = win ? win_rel(i, j, ox, oy, Ny) : -1;
            if (d00 >= 0) {
              const unsigned int xy = wx1 * wy1;  // < 2^32
              atomicAdd(&Cn[d00], 1u);
              if (wx1) atomicAdd(&Cx[d00], wx1);
              if (wy1) atomicAdd(&Cy[d00], wy1);
              if (xy >> 16) atomicAdd(&Ch[d00], xy >> 16);
              if (xy & 0xFFFFu) atomicAdd(&Cl[d00], xy & 0xFFFFu);
            } else {
              deposit2_global(D, xn, yn, sign);
            }
          }
        }
        store4(xs + base, xv);
        store4(us + base, uv);
        store4(ys + base, yv);
        store4(ws + base, wv);
      }
    }
    if (win) {  // flush the deposit window into the int64 grid
      __syncthreads();
      for (int q = threadIdx.x; q < kW2 * kW2; q += kThreads2) {
        const int p = q / kW2, r = q % kW2;
        constexpr long long A = 65536;
        auto sxy = [&](int c) { return (static_cast<long long>(Ch[c]) << 16) + static_cast<long long>(Cl[c]); };
        // w00 of cell (p, r), w10 of (p-1, r), w01 of (p, r-1), w11 of (p-1, r-1)
        long long v = A * A * static_cast<long long>(Cn[q]) - A * static_cast<long long>(Cx[q]) -
                      A * static_cast<long long>(Cy[q]) + sxy(q);
        if (p > 0) v += A * static_cast<long long>(Cx[q - kW2]) - sxy(q - kW2);
        if (r > 0) v += A * static_cast<long long>(Cy[q - 1]) - sxy(q - 1);
        if (p > 0 && r > 0) v += sxy(q - kW2 - 1);
        if (v == 0) continue;
        const int gx = ox + q / kW2;
        const int gy = wrapi(oy + q % kW2, Ny);
        const long long dbl = (gx == 0 || gx == D.Nx) ? 2 : 1;
        atomic_add_i64(&D.G2[static_cast<long long>(gx) * Ny + gy], sign * dbl * static_cast<long long>(v));
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&item_ctr[1], 1) == static_cast<int>(gridDim.x) - 1) {  // every CTA has left the queue
      item_ctr[0] = 0;
      item_ctr[1] = 0;
      __threadfence();
    }
  }
  // tallies of the absorbed particles
  for (int e = 0; e < 2; ++e)
    for (int s = 0; s < kSpecies; ++s) {
      const unsigned int v = warp_sum_u(a_cnt[e][s]);
      if (lane_id() == 0 && v) atomicAdd(&s_cnt[e][s], static_cast<unsigned long long>(v));
    }
  cfl = warp_max_u(cfl);
  if (lane_id() == 0 && cfl) atomicMax(&s_cfl, cfl);
  __syncthreads();

  // --- secondary emission from the ions this CTA saw absorbed ---------------
  const int na = min(s_abs_n, abs_cap);
  const double dx = P->dx, dt = P->dt, dy = D.dy;
  for (int r = threadIdx.x; r < na; r += kThreads2) {
    const AbsRec2 rec = my_abs[r];
    const double vx = static_cast<double>(rec.u) * dx / dt;
    const double vy = static_cast<double>(rec.w) * dy / dt;
    const double Eev = 0.5 * P->m_i * (vx * vx + vy * vy) / P->e;
    const int nse = see_count(P, Eev, rec.id, step);
    const int el = static_cast<int>(rec.el);
    if (el == 0) {
      atomicAdd(reinterpret_cast<unsigned long long*>(&s_energy),
                static_cast<unsigned long long>(__double2ll_rn(Eev * 256.0)));
      if (nse) atomicAdd(reinterpret_cast<unsigned long long*>(&s_conv),
                         static_cast<unsigned long long>(static_cast<long long>(nse)));
    }
    if (nse == 0) continue;
    atomicAdd(&s_emit[el], static_cast<unsigned long long>(nse));
    const unsigned long long wb =
        atomicAdd(reinterpret_cast<unsigned long long*>(&S->n_alloc[CP_SECONDARIES]),
                  static_cast<unsigned long long>(nse));
    float* xs = reinterpret_cast<float*>(S->xi[CP_SECONDARIES]);
    float* us = reinterpret_cast<float*>(S->u[CP_SECONDARIES]);
    float* ys = reinterpret_cast<float*>(Dp->y[CP_SECONDARIES]);
    float* ws = reinterpret_cast<float*>(Dp->w[CP_SECONDARIES]);
    for (int jn = 0; jn < nse; ++jn) {
      double frac;
      const double use = see_speed(P, rec.id, step, jn, &frac) * dt / dx;
      const double xd = (el == 0) ? __dmul_rn(use, frac) : __dsub_rn(static_cast<double>(D.Nx), __dmul_rn(use, frac));
      const float xr = nudge_inside<float>(xd, D.Nx);
      const unsigned long long slot = wb + static_cast<unsigned long long>(jn);
      if (slot < static_cast<unsigned long long>(P->cap[CP_SECONDARIES])) {
        xs[slot] = xr;
        us[slot] = static_cast<float>(el == 0 ? use : -use);
        ys[slot] = rec.eta;
        ws[slot] = 0.0f;
        deposit2_global(D, xr, rec.eta, -1LL);
      } else {
        s_over = 1;
      }
    }
  }

  // --- beam ions entering at x = d with a Gaussian transverse profile --------
  const int Bn = P->beam_per_step;
  if (Bn > 0) {
    float* xs = reinterpret_cast<float*>(S->xi[CP_IONS]);
    float* us = reinterpret_cast<float*>(S->u[CP_IONS]);
    float* ys = reinterpret_cast<float*>(Dp->y[CP_IONS]);
    float* ws = reinterpret_cast<float*>(Dp->w[CP_IONS]);
    uint32_t* idw = S->id;
    const uint32_t id0 = S->beam_id_base;
    const double pi = 3.14159265358979323846;
    for (int k0 = blockIdx.x * kThreads2; k0 < Bn; k0 += gridDim.x * kThreads2) {
      const int k = k0 + threadIdx.x;
      const bool act = k < Bn;
      const unsigned ball = __ballot_sync(0xffffffffu, act);
      unsigned long long wbase = 0ULL;
      if (lane_id() == 0 && ball)
        wbase = atomicAdd(reinterpret_cast<unsigned long long*>(&S->n_alloc[CP_IONS]),
                          static_cast<unsigned long long>(__popc(ball)));
      wbase = __shfl_sync(0xffffffffu, wbase, 0);
      if (!act) continue;
      const U64x4 wv = philox4x64_10(static_cast<uint64_t>(k), static_cast<uint64_t>(step), 0, 0,
                                     P->seed, kTagBeam);
      const double frac = u01(wv.w[0]);
      const double Eb = (P->beam_mode == 0)
                            ? P->beam_E_eV
                            : __dadd_rn(P->beam_Emin_eV, __dmul_rn(__dsub_rn(P->beam_Emax_eV, P->beam_Emin_eV), u01(wv.w[1])));
      const double ub = sqrt(2.0 * Eb * P->e / P->m_i) * dt / dx;
      const double z = sqrt(-2.0 * log(u01(wv.w[2]))) * cos(2.0 * pi * u01(wv.w[3]));
      double yc = D.beam_yc + D.beam_sigma * z;
      yc -= static_cast<double>(Ny) * floor(yc / static_cast<double>(Ny));
      float yr = static_cast<float>(yc);
      if (!(yr < D.Nyf)) yr = 0.0f;
      const float xr = nudge_inside<float>(__dsub_rn(static_cast<double>(D.Nx), __dmul_rn(ub, frac)), D.Nx);
      const unsigned long long slot =
          wbase + static_cast<unsigned long long>(__popc(ball & ((1u << lane_id()) - 1u)));
      if (slot < static_cast<unsigned long long>(P->cap[CP_IONS])) {
        xs[slot] = xr;
        us[slot] = static_cast<float>(-ub);
        ys[slot] = yr;
        ws[slot] = 0.0f;
        idw[slot] = id0 + static_cast<uint32_t>(step * Bn + k);
        deposit2_global(D, xr, yr, 1LL);
      } else {
        s_over = 1;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int e = 0; e < 2; ++e)
      for (int s = 0; s < kSpecies; ++s)
        if (s_cnt[e][s]) atomicAdd(&S->absorbed[e][s], s_cnt[e][s]);
    if (s_emit[0]) atomicAdd(&S->emitted[0], s_emit[0]);
    if (s_emit[1]) atomicAdd(&S->emitted[1], s_emit[1]);
    const long long conv = static_cast<long long>(s_cnt[0][CP_IONS]) -
                           static_cast<long long>(s_cnt[0][CP_ELECTRONS]) -
                           static_cast<long long>(s_cnt[0][CP_SECONDARIES]) + s_conv;
    if (conv) atomic_add_i64(&S->conv_count, conv);
    if (s_energy) atomic_add_i64(&S->ion_energy_q, s_energy);
    if (s_cfl) atomicMax(&S->max_cfl_bits, s_cfl);
    if (blockIdx.x == 0 && Bn > 0) atomicAdd(&S->injected, static_cast<unsigned long long>(Bn));
    if (s_over || s_abs_n > abs_cap) atomicCAS(&S->status, 0, CP_ERR_CAPACITY);
  }
}

// Level 0: deposit every live particle of one species (global atomics).
__global__ void k2_deposit0(const DevState* S, const Dev2D* Dp, int s) {
  const Dev2D& D = *Dp;
  const float* xs = reinterpret_cast<const float*>(S->xi[s]);
  const float* ys = reinterpret_cast<const float*>(D.y[s]);
  const long long n = S->n_proc[s];
  const long long sign = (s == CP_IONS) ? 1LL : -1LL;
  for (long long k = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; k < n;
       k += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float x = xs[k];
    if (x > 0.0f && x < D.Nxf) deposit2_global(D, x, ys[k], sign);
  }
}

// ---------------------------------------------------------------------------
// Counting sort by tile (drops dead slots; tile segments padded to 4)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int tile_of(const Dev2D& D, float x, float y) {
  const int tx = min(static_cast<int>(x) / kT2, D.ntx - 1);
  const int ty = min(static_cast<int>(y) / kT2, D.nty - 1);
  return tx * D.nty + ty;
}

// Counting sort in three passes, each block owning one contiguous range of
// slots: per-block tile histograms, then (one block) the tile segments and
// every block's base in each tile, then the scatter with shared-memory
// cursors -- no global atomics on the per-tile cursors.
__device__ __forceinline__ void block_range(long long n, long long* b0, long long* b1) {
  *b0 = n * blockIdx.x / gridDim.x;
  *b1 = n * (blockIdx.x + 1) / gridDim.x;
}

__global__ void k2_hist(const DevState* S, Dev2D* Dp, int s) {
  extern __shared__ int hist[];
  const Dev2D& D = *Dp;
  for (int t = threadIdx.x; t < D.T; t += blockDim.x) hist[t] = 0;
  __syncthreads();
  const float* xs = reinterpret_cast<const float*>(S->xi[s]);
  const float* ys = reinterpret_cast<const float*>(D.y[s]);
  long long b0, b1;
  block_range(S->n_proc[s], &b0, &b1);
  // warp-uniform trips; each run of consecutive lanes in one tile (sorted
  // data: most of a warp) is counted by one shared-memory atomic
  constexpr int U = 4;
  const long long step = static_cast<long long>(blockDim.x) * U;
  for (long long k0 = b0 + (threadIdx.x & ~31u); k0 < b1; k0 += step) {
    float x[U], y[U];
#pragma unroll
    for (int c = 0; c < U; ++c) {
      const long long k = k0 + static_cast<long long>(c) * blockDim.x + lane_id();
      const bool in = k < b1;
      x[c] = in ? xs[k] : -1.0f;
      y[c] = in ? ys[k] : 0.0f;
    }
#pragma unroll
    for (int c = 0; c < U; ++c) {
      const int t = (x[c] > 0.0f && x[c] < D.Nxf) ? tile_of(D, x[c], y[c]) : -1;
      const int tp = __shfl_up_sync(0xffffffffu, t, 1);
      const bool start = (lane_id() == 0) || (t != tp);
      const unsigned starts = __ballot_sync(0xffffffffu, start);
      const unsigned later = starts & ~((2u << lane_id()) - 1u);
      const int next = later ? __ffs(later) - 1 : 32;
      if (start && t >= 0) atomicAdd(&hist[t], next - static_cast<int>(lane_id()));
    }
  }
  __syncthreads();
  const int G = gridDim.x;  // layout [tile][block]: each tile's counts contiguous
  for (int t = threadIdx.x; t < D.T; t += blockDim.x) D.bhist[static_cast<long long>(t) * G + blockIdx.x] = hist[t];
}

// one block: tile totals and per-block offsets, tile segment starts (padded
// to 4), work-item prefix, dead padding in the destination, block bases
__global__ void k2_scan(DevState* S, Dev2D* Dp, int s, int G) {
  Dev2D& D = *Dp;
  __shared__ int wsum[32], wsum2[32];
  const int T = D.T;
  int* cnt = D.tile_cnt + s * T;
  int* ts = D.tile_start + s * (T + 1);
  int* wo = D.wi_off + s * (T + 1);
  (void)G;
  const int per = (T + blockDim.x - 1) / blockDim.x;
  const int t0 = min(static_cast<int>(threadIdx.x) * per, T), t1 = min(t0 + per, T);
  int a = 0, bq = 0;
  for (int t = t0; t < t1; ++t) {
    a += (cnt[t] + 3) & ~3;
    bq += (cnt[t] + kChunk2 - 1) / kChunk2;
  }
  int ia = a, ib = bq;
  for (int o = 1; o < 32; o <<= 1) {
    const int ya = __shfl_up_sync(0xffffffffu, ia, o), yb = __shfl_up_sync(0xffffffffu, ib, o);
    if (static_cast<int>(lane_id()) >= o) {
      ia += ya;
      ib += yb;
    }
  }
  const int w = threadIdx.x >> 5;
  if (lane_id() == 31) {
    wsum[w] = ia;
    wsum2[w] = ib;
  }
  __syncthreads();
  int ba = 0, bb = 0;
  for (int q = 0; q < w; ++q) {
    ba += wsum[q];
    bb += wsum2[q];
  }
  int ra = ba + ia - a, rb = bb + ib - bq;
  float* xd = reinterpret_cast<float*>(S->xi_alt[s]);
  float* ud = reinterpret_cast<float*>(S->u_alt[s]);
  const long long cap = D.cap[s];
  for (int t = t0; t < t1; ++t) {
    ts[t] = ra;
    wo[t] = rb;
    const int c = cnt[t], c4 = (c + 3) & ~3;
    for (int k = c; k < c4; ++k) {  // dead padding slots
      if (ra + k < cap) {
        xd[ra + k] = -1.0f;
        ud[ra + k] = 0.0f;
      }
    }
    ra += c4;
    rb += (c + kChunk2 - 1) / kChunk2;
  }
  if (threadIdx.x == blockDim.x - 1) {
    ts[T] = ra;
    wo[T] = rb;
  }
}

// one block per tile: exclusive scan of the per-block counts over the blocks
// (each block's offset within the tile) and the tile's total
__global__ void k2_tilescan(Dev2D* Dp, int s, int G) {
  Dev2D& D = *Dp;
  __shared__ int wsum[32];
  const int t = blockIdx.x, T = D.T;
  const int per = (G + blockDim.x - 1) / blockDim.x;
  const int b0 = min(static_cast<int>(threadIdx.x) * per, G), b1 = min(b0 + per, G);
  int* col = D.bhist + static_cast<long long>(t) * G;
  int loc = 0;
  for (int b = b0; b < b1; ++b) loc += col[b];
  int incl = loc;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (static_cast<int>(lane_id()) >= o) incl += y;
  }
  const int w = threadIdx.x >> 5;
  if (lane_id() == 31) wsum[w] = incl;
  __syncthreads();
  int base = 0;
  for (int q = 0; q < w; ++q) base += wsum[q];
  int run = base + incl - loc;
  for (int b = b0; b < b1; ++b) {
    const int c = col[b];
    col[b] = run;
    run += c;
  }
  if (threadIdx.x == blockDim.x - 1) D.tile_cnt[s * T + t] = base + incl;
}

// block bases: tile start + the block's offset within the tile
__global__ void k2_bases(Dev2D* Dp, int s, int G) {
  Dev2D& D = *Dp;
  const long long n = static_cast<long long>(G) * D.T;
  const int* ts = D.tile_start + s * (D.T + 1);
  for (long long q = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; q < n;
       q += static_cast<long long>(gridDim.x) * blockDim.x)
    D.bhist[q] += ts[q / G];
}

__global__ void __launch_bounds__(512, 2) k2_scatter(const DevState* S, Dev2D* Dp, int s) {
  extern __shared__ int cur[];
  const Dev2D& D = *Dp;
  for (int t = threadIdx.x; t < D.T; t += blockDim.x)
    cur[t] = D.bhist[static_cast<long long>(t) * gridDim.x + blockIdx.x];
  __syncthreads();
  const float* xs = reinterpret_cast<const float*>(S->xi[s]);
  const float* us = reinterpret_cast<const float*>(S->u[s]);
  const float* ys = reinterpret_cast<const float*>(D.y[s]);
  const float* ws = reinterpret_cast<const float*>(D.w[s]);
  float* xd = reinterpret_cast<float*>(S->xi_alt[s]);
  float* ud = reinterpret_cast<float*>(S->u_alt[s]);
  float* yd = reinterpret_cast<float*>(D.y_alt[s]);
  float* wd = reinterpret_cast<float*>(D.w_alt[s]);
  const uint32_t* is = S->id;
  uint32_t* id_d = S->id_alt;
  const bool ions = (s == CP_IONS);
  long long b0, b1;
  block_range(S->n_proc[s], &b0, &b1);
  constexpr int U = 2;  // warp chunks whose loads are issued together
  const long long step = static_cast<long long>(blockDim.x) * U;
  for (long long k0 = b0 + (threadIdx.x & ~31u); k0 < b1; k0 += step) {
    float x[U], y[U], u[U], w[U];
    uint32_t id[U];
#pragma unroll
    for (int c = 0; c < U; ++c) {  // every load first: one memory round trip per U chunks
      const long long k = k0 + static_cast<long long>(c) * blockDim.x + lane_id();
      const bool in = k < b1;
      x[c] = in ? xs[k] : -1.0f;
      y[c] = in ? ys[k] : 0.0f;
      u[c] = in ? us[k] : 0.0f;
      w[c] = in ? ws[k] : 0.0f;
      id[c] = (in && ions) ? is[k] : 0u;
    }
#pragma unroll
    for (int c = 0; c < U; ++c) {
      const int t = (x[c] > 0.0f && x[c] < D.Nxf) ? tile_of(D, x[c], y[c]) : -1;
      // runs of consecutive lanes in one tile: the run's first lane reserves
      // its length, every lane takes the slot of its place in the run
      const int tp = __shfl_up_sync(0xffffffffu, t, 1);
      const bool start = (lane_id() == 0) || (t != tp);
      const unsigned starts = __ballot_sync(0xffffffffu, start);
      const unsigned later = starts & ~((2u << lane_id()) - 1u);  // run starts after this lane
      const int next = later ? __ffs(later) - 1 : 32;
      const int rs = 31 - __clz(starts & ((2u << lane_id()) - 1u));  // this lane's run start
      int base = 0;
      if (start && t >= 0) base = atomicAdd(&cur[t], next - static_cast<int>(lane_id()));
      base = __shfl_sync(0xffffffffu, base, rs);
      if (t < 0) continue;
      const long long o = static_cast<long long>(base) + (static_cast<int>(lane_id()) - rs);
      if (o >= D.cap[s]) continue;  // the sorted store would not fit (reported by k2_swap)
      xd[o] = x[c];
      ud[o] = u[c];
      yd[o] = y[c];
      wd[o] = w[c];
      if (ions) id_d[o] = id[c];
    }
  }
}

// swap the sorted buffers in; one thread
__global__ void k2_swap(DevState* S, Dev2D* Dp, int s) {
  Dev2D& D = *Dp;
  void* t;
  t = S->xi[s]; S->xi[s] = S->xi_alt[s]; S->xi_alt[s] = t;
  t = S->u[s]; S->u[s] = S->u_alt[s]; S->u_alt[s] = t;
  t = D.y[s]; D.y[s] = D.y_alt[s]; D.y_alt[s] = t;
  t = D.w[s]; D.w[s] = D.w_alt[s]; D.w_alt[s] = t;
  if (s == CP_IONS) {
    uint32_t* ti = S->id;
    S->id = S->id_alt;
    S->id_alt = ti;
  }
  long long n = D.tile_start[s * (D.T + 1) + D.T];
  if (n > D.cap[s]) {
    n = D.cap[s] & ~3LL;
    atomicCAS(&S->status, 0, CP_ERR_CAPACITY);
  }
  D.n_sorted[s] = n;
  S->n_alloc[s] = n;
  S->n_proc[s] = n;
}

// ---------------------------------------------------------------------------
// Transverse transforms
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-place radix-2 FFT of buf[0..n) (input in bit-reversed order), sign -1
// forward (twiddles tw[k] = exp(-2 pi i k/n)), +1 inverse (conjugates).
__device__ void fft_radix2(float2* buf, const float2* __restrict__ tw, int n, int inverse) {
  for (int half = 1; half < n; half <<= 1) {
    const int stride = n / (2 * half);
    for (int b = threadIdx.x; b < n / 2; b += blockDim.x) {
      const int grp = b / half, pos = b % half;
      const int i0 = grp * 2 * half + pos, i1 = i0 + half;
      float2 w = tw[pos * stride];
      if (inverse) w.y = -w.y;
      const float2 u = buf[i0], v = cmul(buf[i1], w);
      buf[i0] = make_float2(u.x + v.x, u.y + v.y);
      buf[i1] = make_float2(u.x - v.x, u.y - v.y);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int bitrev(int k, int logn) { return static_cast<int>(__brev(static_cast<unsigned>(k)) >> (32 - logn)); }

// row i: exact row sum into the 1D grid, copy and clear, spectrum of the
// fluctuation (rows 1..Nx-1)
__global__ void k2_fwd(Dev2D* Dp, long long* G1) {
  extern __shared__ float2 buf[];
  __shared__ long long wsum[32];
  __shared__ long long s_tot;
  const Dev2D& D = *Dp;
  cudaGridDependencySynchronize();
  const int i = blockIdx.x;
  const int Ny = D.Ny;
  long long* row = D.G2 + static_cast<long long>(i) * Ny;
  long long* last = D.G2last + static_cast<long long>(i) * Ny;
  long long acc = 0;
  for (int j = threadIdx.x; j < Ny; j += blockDim.x) acc += row[j];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane_id() == 0) wsum[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long tot = 0;
    for (int q = 0; q < static_cast<int>(blockDim.x >> 5); ++q) tot += wsum[q];
    s_tot = tot;
    G1[i] = tot;
  }
  __syncthreads();
  const long long tot = s_tot;
  const double mean = static_cast<double>(tot) / static_cast<double>(Ny);
  const bool interior = (i > 0 && i < D.Nx);
  for (int j = threadIdx.x; j < Ny; j += blockDim.x) {
    const long long g = row[j];
    last[j] = g;
    row[j] = 0;
    if (interior)
      buf[bitrev(j, D.logNy)] =
          make_float2(static_cast<float>((static_cast<double>(g) - mean) * D.rho_scale), 0.0f);
  }
  __syncthreads();
  if (!interior) return;
  fft_radix2(buf, D.tw, Ny, 0);
  float2* R = D.R + static_cast<long long>(i) * (Ny / 2 + 1);
  for (int k = threadIdx.x; k <= Ny / 2; k += blockDim.x) R[k] = buf[k];
}

// One warp per mode k = 1..Ny/2: Thomas over i = 1..Nx-1 with phi = 0 at
// both ends for  Phi_{i-1} - (2 + kappa_k) Phi_i + Phi_{i+1} = -dx^2 R_i / eps0.
// The elimination factors depend on (i, k) only and are tabulated once
// (k2_tables).  Both substitutions are first-order linear recurrences,
// d_i = a_i d_{i-1} + b_i (a_i = -inv_i, b_i = c inv_i R_i) forward and
// x_i = -c'_i x_{i+1} + d_i backward; each lane composes the affine map of
// its segment of rows, a warp scan of the maps gives every segment its
// incoming value, and the lanes then apply their segments.
struct Aff {
  float a;
  float2 b;
};

__device__ __forceinline__ Aff aff_then(Aff f, Aff g) {  // g after f
  Aff h;
  h.a = g.a * f.a;
  h.b = make_float2(fmaf(g.a, f.b.x, g.b.x), fmaf(g.a, f.b.y, g.b.y));
  return h;
}

__device__ __forceinline__ Aff aff_shfl_up(Aff f, int o) {
  Aff r;
  r.a = __shfl_up_sync(0xffffffffu, f.a, o);
  r.b.x = __shfl_up_sync(0xffffffffu, f.b.x, o);
  r.b.y = __shfl_up_sync(0xffffffffu, f.b.y, o);
  return r;
}

constexpr int kU2 = 8;  // rows of loads issued ahead

__global__ void __launch_bounds__(128) k2_modes(Dev2D* Dp, float c_rhs) {
  const Dev2D& D = *Dp;
  const int k = 1 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int M = D.Ny / 2 + 1;
  if (k >= M) return;  // whole warps leave together
  const int lane = static_cast<int>(lane_id());
  float2* __restrict__ R = D.R;
  const float* __restrict__ inv = D.tinv;
  const float* __restrict__ cp = D.cp;
  const int n = D.Nx - 1;             // rows 1..n
  const int seg = (n + 31) / 32;
  const int r0 = 1 + lane * seg, r1 = min(n + 1, r0 + seg);  // this lane's rows [r0, r1)
  // forward: compose this segment's map
  Aff f;
  f.a = 1.0f;
  f.b = make_float2(0.0f, 0.0f);
  for (int i0 = r0; i0 < r1; i0 += kU2) {
    float2 rr[kU2];
    float iv[kU2];
#pragma unroll
    for (int q = 0; q < kU2; ++q)
      if (i0 + q < r1) {
        rr[q] = R[static_cast<long long>(i0 + q) * M + k];
        iv[q] = inv[static_cast<long long>(i0 + q) * M + k];
      }
#pragma unroll
    for (int q = 0; q < kU2; ++q)
      if (i0 + q < r1) {
        Aff g;
        g.a = -iv[q];
        g.b = make_float2(c_rhs * iv[q] * rr[q].x, c_rhs * iv[q] * rr[q].y);
        f = aff_then(f, g);
      }
  }
  // exclusive scan over the lanes: the map from d_0 = 0 to this segment's start
  Aff incl = f;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const Aff y = aff_shfl_up(incl, o);
    if (lane >= o) incl = aff_then(y, incl);
  }
  Aff ex = aff_shfl_up(incl, 1);
  float2 d = (lane == 0) ? make_float2(0.0f, 0.0f) : ex.b;
  // forward: apply
  for (int i0 = r0; i0 < r1; i0 += kU2) {
    float2 rr[kU2];
    float iv[kU2];
#pragma unroll
    for (int q = 0; q < kU2; ++q)
      if (i0 + q < r1) {
        rr[q] = R[static_cast<long long>(i0 + q) * M + k];
        iv[q] = inv[static_cast<long long>(i0 + q) * M + k];
      }
#pragma unroll
    for (int q = 0; q < kU2; ++q)
      if (i0 + q < r1) {
        const float a = -iv[q];
        d = make_float2(fmaf(a, d.x, c_rhs * iv[q] * rr[q].x), fmaf(a, d.y, c_rhs * iv[q] * rr[q].y));
        R[static_cast<long long>(i0 + q) * M + k] = d;
      }
  }
  // backward: x_i = -c'_i x_{i+1} + d_i, segments from the last row down
  Aff g;
  g.a = 1.0f;
  g.b = make_float2(0.0f, 0.0f);
  for (int i0 = r1 - 1; i0 >= r0; i0 -= kU2) {
    float2 dd[kU2];
    float cc[kU2];
#pragma unroll
    for (int q = 0; q < kU2; ++q)
      if (i0 - q >= r0) {
        dd[q] = R[static_cast<long long>(i0 - q) * M + k];
        cc[q] = cp[static_cast<long long>(i0 - q) * M + k];
      }
#pragma unroll
    for (int q = 0; q < kU2; ++q)
      if (i0 - q >= r0) {
        Aff h;
        h.a = -cc[q];
        h.b = dd[q];
        g = aff_then(g, h);
      }
  }
  // reverse exclusive scan (lane 31 holds the last rows)
  Aff incl2 = g;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    Aff y;
    y.a = __shfl_down_sync(0xffffffffu, incl2.a, o);
    y.b.x = __shfl_down_sync(0xffffffffu, incl2.b.x, o);
    y.b.y = __shfl_down_sync(0xffffffffu, incl2.b.y, o);
    if (lane + o < 32) incl2 = aff_then(y, incl2);
  }
  float2 x;
  {
    const float bx = __shfl_down_sync(0xffffffffu, incl2.b.x, 1);
    const float by = __shfl_down_sync(0xffffffffu, incl2.b.y, 1);
    x = (lane == 31) ? make_float2(0.0f, 0.0f) : make_float2(bx, by);
  }
  for (int i0 = r1 - 1; i0 >= r0; i0 -= kU2) {
    float2 dd[kU2];
    float cc[kU2];
#pragma unroll
    for (int q = 0; q < kU2; ++q)
      if (i0 - q >= r0) {
        dd[q] = R[static_cast<long long>(i0 - q) * M + k];
        cc[q] = cp[static_cast<long long>(i0 - q) * M + k];
      }
#pragma unroll
    for (int q = 0; q < kU2; ++q)
      if (i0 - q >= r0) {
        x = make_float2(fmaf(-cc[q], x.x, dd[q].x), fmaf(-cc[q], x.y, dd[q].y));
        R[static_cast<long long>(i0 - q) * M + k] = x;
      }
  }
}

// row i = 1..Nx-1: inverse transform of the mode solution -> phit
__global__ void k2_inv(Dev2D* Dp) {
  extern __shared__ float2 buf[];
  const Dev2D& D = *Dp;
  const int i = 1 + blockIdx.x;
  const int Ny = D.Ny, M = Ny / 2 + 1;
  const float2* R = D.R + static_cast<long long>(i) * M;
  for (int k = threadIdx.x; k < Ny; k += blockDim.x) {
    float2 v;
    if (k == 0) v = make_float2(0.0f, 0.0f);
    else if (k < M) v = R[k];
    else {
      const float2 c = R[Ny - k];
      v = make_float2(c.x, -c.y);
    }
    if (k == Ny / 2) v.y = 0.0f;
    buf[bitrev(k, D.logNy)] = v;
  }
  __syncthreads();
  fft_radix2(buf, D.tw, Ny, 1);
  const float inv_n = 1.0f / static_cast<float>(Ny);
  float* out = D.phit + static_cast<long long>(i) * Ny;
  for (int j = threadIdx.x; j < Ny; j += blockDim.x) out[j] = buf[j].x * inv_n;
}

// E_x = E_0(x) + (phit_ij - phit_i+1,j)/dx, E_y = (phit_ij - phit_i,j+1)/dy
__global__ void k2_fields(Dev2D* Dp, const double* __restrict__ E64) {
  const Dev2D& D = *Dp;
  const int Ny = D.Ny;
  const long long n = static_cast<long long>(D.Nx + 1) * Ny;
  for (long long q = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; q < n;
       q += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(q / Ny), j = static_cast<int>(q % Ny);
    const float p = D.phit[q];
    if (i < D.Nx)
      D.Ex[q] = static_cast<float>(E64[i]) + (p - D.phit[q + Ny]) * D.inv_dx;
    const int j1 = (j + 1 == Ny) ? 0 : j + 1;
    D.Ey[q] = (p - D.phit[static_cast<long long>(i) * Ny + j1]) * D.inv_dy;
  }
}

__global__ void k2_tables(Dev2D* Dp, double r2) {
  Dev2D& D = *Dp;
  const int Ny = D.Ny, M = Ny / 2 + 1;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
    double sn, cs;
    sincospi(2.0 * k / Ny, &sn, &cs);
    const double kap = r2 * (2.0 - 2.0 * cs);
    D.kappa[k] = static_cast<float>(kap);
    if (k < Ny / 2) D.tw[k] = make_float2(static_cast<float>(cs), static_cast<float>(-sn));
    // Thomas elimination of mode k: inv_i = 1/(b - c'_{i-1}), c'_i = inv_i (last row 0)
    const double bk = -(2.0 + kap);
    double cprev = 0.0;
    for (int i = 1; i < D.Nx; ++i) {
      const double iv = 1.0 / (bk - cprev);
      const double c = (i + 1 < D.Nx) ? iv : 0.0;
      D.tinv[static_cast<long long>(i) * M + k] = static_cast<float>(iv);
      D.cp[static_cast<long long>(i) * M + k] = static_cast<float>(c);
      cprev = c;
    }
  }
}

// ---------------------------------------------------------------------------
// Host-side launchers
// ---------------------------------------------------------------------------
size_t dev2d_bytes() { return sizeof(Dev2D); }
size_t absrec2_bytes() { return sizeof(AbsRec2); }
int kchunk2() { return kChunk2; }
int tile2() { return kT2; }

constexpr size_t kCwinBytes = 5 * sizeof(unsigned int) * kW2 * kW2;  // the deposit window's cell sums

cudaError_t push2_occupancy(int* per_sm) {
  const cudaError_t e = cudaFuncSetAttribute(k2_push, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(kCwinBytes));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k2_push, kThreads2, kCwinBytes);
}

cudaError_t push2_launch(const DevParams* P, DevState* S, void* D, const void* D_host, void* abs,
                         int abs_cap, int grid, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(kThreads2, 1, 1);
  cfg.dynamicSmemBytes = kCwinBytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k2_push, P, S, static_cast<const Dev2D*>(D),
                            *static_cast<const Dev2D*>(D_host), static_cast<Dev2D*>(D)->item_ctr,
                            static_cast<AbsRec2*>(abs), abs_cap);
}

cudaError_t sort2_launch(DevState* S, void* D, int T, int s, int sms, cudaStream_t st) {
  Dev2D* Dp = static_cast<Dev2D*>(D);
  const size_t hs = sizeof(int) * T;
  const int G = 2 * sms;  // must match the blocks the per-block histograms were sized for
  k2_hist<<<G, 512, hs, st>>>(S, Dp, s);
  k2_tilescan<<<T, 128, 0, st>>>(Dp, s, G);
  k2_scan<<<1, 1024, 0, st>>>(S, Dp, s, G);
  k2_bases<<<std::min(4096, (G * T + 255) / 256), 256, 0, st>>>(Dp, s, G);
  k2_scatter<<<G, 512, hs, st>>>(S, Dp, s);
  k2_swap<<<1, 1, 0, st>>>(S, Dp, s);
  return cudaGetLastError();
}

cudaError_t solve2_fwd_launch(void* D, long long* G1, int Nx, int Ny, cudaStream_t st) {
  const size_t smem = sizeof(float2) * Ny;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(Nx + 1, 1, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k2_fwd, static_cast<Dev2D*>(D), G1);
}

cudaError_t solve2_modes_launch(void* D, int Nx, int Ny, float c_rhs, const double* E64,
                                cudaStream_t st) {
  Dev2D* Dp = static_cast<Dev2D*>(D);
  const int M = Ny / 2;
  k2_modes<<<(M + 3) / 4, 128, 0, st>>>(Dp, c_rhs);
  if (Nx > 1) k2_inv<<<Nx - 1, 256, sizeof(float2) * Ny, st>>>(Dp);
  const long long n = static_cast<long long>(Nx + 1) * Ny;
  const int grid = static_cast<int>(std::min<long long>((n + 255) / 256, 4096));
  k2_fields<<<grid, 256, 0, st>>>(Dp, E64);
  return cudaGetLastError();
}

cudaError_t deposit2_level0_launch(DevState* S, const void* D, int sms, cudaStream_t st) {
  for (int s = 0; s < kSpecies; ++s)
    k2_deposit0<<<2 * sms, 512, 0, st>>>(S, static_cast<const Dev2D*>(D), s);
  return cudaGetLastError();
}

cudaError_t tables2_launch(void* D, int Ny, double r2, cudaStream_t st) {
  k2_tables<<<(Ny / 2 + 128) / 128, 128, 0, st>>>(static_cast<Dev2D*>(D), r2);
  return cudaGetLastError();
}

}  // namespace cpk
