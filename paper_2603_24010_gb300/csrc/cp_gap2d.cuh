// cp_gap2d.cuh -- device state of the 2D planar gap shared by its kernels
// (cp_gap2d.cu) and the host code that sets it up (cp_api.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "cp_device.cuh"

namespace cpk {

constexpr int kT2 = 32;          // tile edge in cells
constexpr int kH2 = 4;           // halo of the field and deposit windows in cells
constexpr int kW2 = kT2 + 2 * kH2 + 2;  // window edge in nodes (42)
constexpr int kChunk2 = 32768;   // particles per work item
constexpr int kThreads2 = 512;
constexpr double kFix2 = 4294967296.0;  // charge-grid units per macroparticle (2^16 per axis)

struct Dev2D {
  int Nx, Ny, ntx, nty, T;
  int sort_every;
  float Nxf, Nyf;
  float inv_dx, inv_dy;
  float kx[2][kSpecies], ky[2][kSpecies];  // kick factors (half, full)
  double dx, dy, rho_scale;               // rho = G rho_scale
  double beam_sigma, beam_yc;             // in cells
  void* y[kSpecies];
  void* w[kSpecies];
  void* y_alt[kSpecies];
  void* w_alt[kSpecies];
  long long n_sorted[kSpecies];
  long long cap[kSpecies];  // slots of each store
  int* tile_start;  // [3][T+1] particle offsets of the sorted segments
  int* wi_off;      // [3][T+1] prefix of work items per tile
  int* tile_cnt;    // [3][T] live particles per tile (sort scratch)
  int* tile_cur;    // [3][T] scatter cursors
  float* Ex;        // [Nx][Ny]   E_x at (i+1/2, j)
  float* Ey;        // [Nx+1][Ny] E_y at (i, j+1/2)
  long long* G2;    // [Nx+1][Ny] charge being deposited
  long long* G2last;
  float2* R;        // [Nx+1][Ny/2+1] transverse spectra
  float* cp;        // [Nx+1][Ny/2+1] Thomas factors c'_i of each mode
  float* tinv;      // [Nx+1][Ny/2+1] Thomas factors 1/(b - c'_{i-1}) of each mode
  int* bhist;       // [sort blocks][T] per-block tile counts, then bases
  float* phit;      // [Nx+1][Ny] potential of the k != 0 modes
  float* kappa;     // [Ny/2+1] (dx/dy)^2 (2 - 2 cos 2 pi k/Ny)
  float2* tw;       // [Ny/2] exp(-2 pi i k/Ny)
  int logNy;
  int use_win;      // 0 when Ny < the window edge (the window would wrap onto itself)
  int item_ctr[2];  // k2_push's work-item queue: next item, CTAs done (zero between launches)
};

struct AbsRec2 {
  uint32_t id;
  uint32_t el;
  float u, w, eta, pad;
};

}  // namespace cpk
