// cp_device.cuh -- device-side data layout and helpers of the GB300 PIC step.
//
// Layout in HBM (one gap instance):
//   particle stores, structure of arrays, one pair per species
//     xi[s][cap_s]  position in cell units (float or double)
//     u[s][cap_s]   velocity in cells/step
//     id[cap_ions]  uint32 ion id (keys the SEE draws; read only for impacts)
//   each store has a second buffer used by the periodic removal of absorbed
//   particles; the live buffer pointers live in DevState so that captured
//   CUDA graphs stay valid across swaps.
//   G[N+1]        int64 charge grid being deposited for the next level
//                 (2^16 units per macroparticle charge)
//   Glast[N+1]    int64 charge grid of the current level (read-back copy)
//   Epair[N+1]    gather table of the current level in particle precision:
//                 pair k = (Ep_k, Ep_{k+1} - Ep_k) with Ep_0 = E_{1/2},
//                 Ep_k = E_{k-1/2} (k = 1..N), Ep_{N+1} = E_{N-1/2}
//   phi[N+1], E64[N]  FP64 potential and field of the current level
//   abs[grid*cap] per-CTA lists of ions absorbed in the current push
//   hist[rows]    one cp_diag row per level
//   vs[rows]      source voltage polarity V_s(t_n) per level
//
// A dead (absorbed) particle has xi <= 0; live particles have 0 < xi < N.
#pragma once

#include <cstdint>

#include "../../include/cp.h"

namespace cpk {

constexpr int kSpecies = 3;
constexpr int kThreads = 512;          // threads per CTA of the push kernel
constexpr int kCtasPerSm = 2;          // resident push CTAs per SM
constexpr int kPerThread = 4;          // particles per thread per tile (one 16 B vector for FP32)
constexpr int kTile = kThreads * kPerThread;  // particles per CTA tile
constexpr int kFlushTiles = 31;        // tiles between flushes of the 32-bit cell sums
constexpr int kSolveCtas = 8;          // CTAs (one cluster) of the coupled solve (portable)
constexpr int kSolveCtasMax = 16;      // non-portable cluster size used where the GPU allows it
constexpr int kSolveThreads = 512;
constexpr double kFix = 65536.0;       // fixed-point units per macroparticle charge
constexpr uint64_t kTagSee = 0x5345ULL;
constexpr uint64_t kTagBeam = 0x4245ULL;
constexpr uint64_t kTagInit = 0x4D4C50ULL;  // MLP parameter initialisation draws
constexpr uint64_t kTagLoad = 0x4C4F4144ULL;  // initial plasma load
// predictor network shape and feature window
constexpr int kPredWindow = 8;
constexpr int kPredFeat = 5;
constexpr int kPredIn = kPredWindow * kPredFeat;  // 40
constexpr int kHid = 64;
constexpr int kPredOut = 2;
constexpr int kPredMinEval = 16;  // checked predictions before the first use
constexpr int kSeePoissonMax = 64;  // truncation of the Poisson emission count
constexpr double kPredAvg = 1.0 / 16.0;  // weight of the running error averages

struct DevParams {
  int32_t N;
  int32_t circuit;
  int32_t beam_per_step;
  int32_t beam_mode;
  double d, dx, dt, area, eps0, e, m_e, m_i, weight;
  double R, L, C, V0, f, tau, polarity;
  double gamma_coef, gamma_max, E_ref_eV, see_scale, T_emit_eV;
  double beam_E_eV, beam_Emin_eV, beam_Emax_eV;
  double beam_ub;        // mono-energetic beam speed sqrt(2 E e / m_i) dt / dx [cells/step]
  double beam_c0, beam_c1;  // uniform beam: ub^2 = c0 + c1 u (u uniform in [0, 1)) [cells^2/step^2]
  uint64_t seed;
  double scale;          // rho_i = G_i * scale  [C/m^3]
  double kappa[kSpecies];  // q dt^2 / (m dx): cells/step^2 per V/m
  double see_vth;        // sqrt(e T_emit / m_e)
  double see_ln_mu, see_ln_sigma;  // lognormal SE energy law: ln(E / 1 eV) ~ N(mu, sigma^2)
  double see_v_eV;       // sqrt(2 e / m_e): speed of an electron of 1 eV
  int32_t see_count_law, see_energy_law;
  double a21;            // 9 L / (4 dt^2) + 3 R / (2 dt): BDF2 coefficient of Q^n
  double alpha;          // dx^2 * scale / eps0: b_i = -alpha G_i
  // host-precomputed factors so that the solve divides nothing in FP64
  double g_strict;       // 1 / a21
  double g_weak;         // 1 / (a21 + 1/C)
  double inv_C;          // 1 / C
  double gam_strict;     // g_strict dx / (eps0 A)
  double inv_den_strict; // 1 / (1 + N gam_strict)
  double dx_eps0;        // dx / eps0
  double inv_A, inv_dx, inv_2dt;
  double L4dt2, R2dt;    // L / (4 dt^2), R / (2 dt)
  // Tesla transformer circuit: the new level's loop charges are linear in
  // the 20 history values h (loop charges of levels n-1..n-4):
  //   strict: Q^n = t_Ps h - phi_0 t_ws   (T'^{-1} H and T'^{-1} e4)
  //   weak:   Q^n = t_Pw h + s t_ww       (T^{-1} H and T^{-1} e4, s the
  //           capacitor term of loop 4)
  double t_Ps[5][20], t_ws[5], t_Pw[5][20], t_ww[5];
  double t_Q0[5];        // loop charges before t = 0
  double gam_tesla;      // [T'^{-1}]_44 dx / (eps0 A)
  double inv_den_tesla;  // 1 / (1 + N gam_tesla)
  float kap_f[2][kSpecies];   // kick factors in FP32: [0] half kick, [1] full kick
  double kap_d[2][kSpecies];  // the same in FP64
  int64_t cap[kSpecies];
  int32_t abs_cap;       // absorbed-ion records per CTA
  int32_t precision;
};

// Record of one ion absorbed during the push (SEE input).
struct AbsRec {
  uint32_t id;
  uint32_t electrode;
  double u;
};

struct DevState {
  void* xi[kSpecies];
  void* u[kSpecies];
  uint32_t* id;
  void* xi_alt[kSpecies];
  void* u_alt[kSpecies];
  uint32_t* id_alt;
  int64_t level;
  int32_t pushed;
  int32_t status;        // 0 or a CP_ERR_* code; stepping stops while non-zero
  double sigma;          // sigma_+ at the current level
  double Qh[4];          // Q^{n}, Q^{n-1}, Q^{n-2}, Q^{n-3}
  double Qt[4][5];       // Tesla circuit: loop charges of levels n, n-1, n-2, n-3
  int64_t n_alloc[kSpecies];  // slots in use (dead included); appends reserve here
  int64_t n_proc[kSpecies];   // slots processed by the current push (multiple of 4)
  int64_t n_live[kSpecies];
  // tallies of the push in progress (cleared by the solve)
  unsigned long long absorbed[2][kSpecies];
  unsigned long long emitted[2];
  unsigned long long injected;
  long long conv_count;
  long long ion_energy_q;     // sum of rint(256 E_eV) over ions absorbed at x = 0
  unsigned int max_cfl_bits;  // float bits of max |u| (non-negative floats order as ints)
  double nxt_Vs, nxt_hist;     // source and BDF2 history of the next level
  double phi0_last;           // phi_0 of the current level (weak: capacitor state)
  // learned weak-coupling predictor (evaluated when a network is installed)
  double feat[kPredWindow][kPredFeat];  // raw feature rows of the last 8 levels (a ring)
  int32_t n_feat;             // rows filled (saturates at kPredWindow)
  int32_t feat_pos;           // ring slot the next level's row goes to
  int32_t pred_ready;         // J_pred holds a prediction for the next level
  double J_pred;              // network's J_hat for the next level [C]
  double err_avg, J_avg;      // running averages of |J - J_hat| and |J|
  int64_t n_eval;             // predictions checked against the realised J
  double J_eff;               // J_pred while its tracked error is within bound, else 0
  double pv_phi0, pv_Qsurf;   // phi_0 and Q_surf of the level before the current one
  unsigned long long compact_n[kSpecies];
  unsigned int compact_done;
  uint32_t beam_id_base;
  cp_diag cur;                // diagnostics of the current level
};

// Installed predictor network: BF16 weights (raw bits, W[out][in]), FP32
// biases and scales.
// Whole 16-byte chunks (alignas pads the size): the solve copies it into
// shared memory with 16-byte asynchronous copies.
struct alignas(16) PredNet {
  uint16_t W1[kHid * kPredIn];
  uint16_t W2[kHid * kHid];
  uint16_t W3[kHid * kHid];
  uint16_t W4[kPredOut * kHid];
  float b1[kHid], b2[kHid], b3[kHid], b4[kPredOut];
  float in_scale[kPredFeat];
  float out_scale[kPredOut];
  double bound;
  double inv_in_scale[kPredFeat];  // 1 / in_scale, formed on the host
};
// bytes of a PredNet as allocated and copied (whole 16-byte chunks)
constexpr size_t kPredNetBytes = sizeof(PredNet);
static_assert(kPredNetBytes % 16 == 0, "the network is copied in 16-byte chunks");

struct Bufs {
  const DevParams* P;
  DevState* S;
  long long* G;
  long long* Glast;
  void* Epair;
  double* phi;
  double* E64;
  AbsRec* abs;
  cp_diag* hist;
  int64_t hist_rows;
  const double* vs;  // polarity V_s(t_n) for every level n (filled once at set-up)
  const PredNet* net;  // installed predictor, or null
  int32_t net_in_push;  // 1: the push runs the predictor (FP32 single gap); 0: the solve does
};

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon et al., SC'11): ten rounds of two 64x64->128
// multiplications with Weyl-sequence key bumps.
// ---------------------------------------------------------------------------
struct U64x4 {
  uint64_t w[4];
};

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                               uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += W0;
    k1 += W1;
  }
  U64x4 o;
  o.w[0] = c0;
  o.w[1] = c1;
  o.w[2] = c2;
  o.w[3] = c3;
  return o;
}

// top 52 bits -> (k + 1/2) 2^-52, exact in binary64, strictly inside (0, 1)
__device__ __forceinline__ double u01(uint64_t w) {
  return __dmul_rn(__dadd_rn((double)(w >> 12), 0.5), 1.0 / 4503599627370496.0);
}

}  // namespace cpk
