// cp_mlp.cuh -- device pieces of the weak-coupling predictor network shared
// by the in-solve inference (cp_solve.cu) and the training kernels
// (cp_mlp.cu): BF16 weight decoding, GELU and its derivative.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "cp_device.cuh"

namespace cpk {

// A BF16 value is the top half of an FP32 word: widening is exact.
__device__ __forceinline__ float bf16_bits_to_float(uint16_t b) {
  return __uint_as_float(static_cast<uint32_t>(b) << 16);
}

// GELU in its erf form, x Phi(x) = x (1 + erf(x / sqrt 2)) / 2.
__device__ __forceinline__ float gelu(float x) {
  return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}

// d/dx [x Phi(x)] = Phi(x) + x phi(x), phi the standard normal density.
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) +
         x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// One dense layer for a single input vector in shared memory, all threads of
// the block taking part: 8 lanes per output neuron (OUT * 8 <= blockDim.x),
// each summing every 8th input in FP32, then a 3-step butterfly.  The calls
// of all threads must be uniform (the shuffles name the whole warp).
template <int IN, int OUT, bool ACT>
__device__ __forceinline__ void dense_one(const uint16_t* __restrict__ W, const float* __restrict__ b,
                                          const float* in, float* out) {
  const int o = static_cast<int>(threadIdx.x) >> 3, part = static_cast<int>(threadIdx.x) & 7;
  float acc = 0.0f;
  if (o < OUT) {
#pragma unroll
    for (int k = part; k < IN; k += 8) acc = fmaf(bf16_bits_to_float(W[o * IN + k]), in[k], acc);
  }
  acc += __shfl_xor_sync(0xffffffffu, acc, 4);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  if (o < OUT && part == 0) {
    const float z = acc + b[o];
    out[o] = ACT ? gelu(z) : z;
  }
}

// dense_one split in two: the BF16 weights a thread uses (every 8th input of
// neuron threadIdx.x / 8, from input threadIdx.x % 8 on) are loaded into
// registers first -- all layers' loads in flight together when the weights
// sit in global memory -- and applied later in dense_one's order.
template <int IN>
struct LaneW {
  uint16_t w[IN / 8];
};

template <int IN, int OUT>
__device__ __forceinline__ void lane_weights(const uint16_t* W, LaneW<IN>& r) {
  static_assert(IN % 8 == 0, "8 lanes per neuron");
  const int o = static_cast<int>(threadIdx.x) >> 3, part = static_cast<int>(threadIdx.x) & 7;
#pragma unroll
  for (int q = 0; q < IN / 8; ++q) r.w[q] = (o < OUT) ? W[o * IN + part + 8 * q] : uint16_t(0);
}

template <int IN, int OUT, bool ACT>
__device__ __forceinline__ void dense_lane(const LaneW<IN>& r, float bias, const float* in, float* out) {
  const int o = static_cast<int>(threadIdx.x) >> 3, part = static_cast<int>(threadIdx.x) & 7;
  float acc = 0.0f;
  if (o < OUT) {
#pragma unroll
    for (int q = 0; q < IN / 8; ++q) acc = fmaf(bf16_bits_to_float(r.w[q]), in[part + 8 * q], acc);
  }
  acc += __shfl_xor_sync(0xffffffffu, acc, 4);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  if (o < OUT && part == 0) {
    const float z = acc + bias;
    out[o] = ACT ? gelu(z) : z;
  }
}

// ---------------------------------------------------------------------------
// One level of the learned weak-coupling predictor.  The same code runs in
// the solve (ensemble members, the 2D gap's mean, FP64 gaps) and in the
// idle tail of the next FP32 push of a single gap; both give the same bits.
// ---------------------------------------------------------------------------
struct PredScratch {
  float x[kPredIn];
  float h1[kHid], h2[kHid], h3[kHid];
  float y[kPredOut];
  double row[kPredFeat];
  int full;    // the window holds 8 levels
  int usable;  // the tracked error allows using the next prediction
};

// What the predictor needs of the level n just solved and of its own state
// before the update (read by thread 0 only).
struct PredLevel {
  double Qconv;              // Q_conv^n
  double phi0, phi0_prev;    // phi_0^n, phi_0^{n-1}
  double Qsurf, Qsurf_prev;  // Q_surf^n, Q_surf^{n-1} (rounded products sigma A)
  double Qn, Q1;             // circuit charges Q^n, Q^{n-1}
  double emitted;            // secondaries emitted at x = 0
  double ion_eV;             // energy of the ions absorbed at x = 0 [eV]
  int had_pred;              // a prediction for level n was made
  double J_pred;             // that prediction
  double err_avg, J_avg;     // running averages before this level
  long long n_eval;
  int pos, n_feat;           // ring slot for level n's row, rows filled
};

// Thread 0 checks the prediction for level n against the realised
// J^n = C (phi_0^n - phi_0^{n-1}) - (Q^n - Q^{n-1}) and appends level n's
// feature row to the 8-level ring; once the window is full every thread
// evaluates the network for J_hat of level n+1, and thread 0 stores it with
// its usable value J_eff (J_hat after 16 checks while avg|J - J_hat| <= bound
// avg|J|, else 0).  v_old: window input threadIdx.x (< 35) from the ring's
// older rows.  All threads of the block call this (its barriers and
// shuffles name them).
__device__ __forceinline__ void pred_level(const PredNet* net, double C, DevState* S,
                                           const PredLevel* L, double v_old, PredScratch* sp) {
  // the network's weights, biases and input scales this thread uses
  LaneW<kPredIn> w1;
  LaneW<kHid> w2, w3, w4;
  lane_weights<kPredIn, kHid>(net->W1, w1);
  lane_weights<kHid, kHid>(net->W2, w2);
  lane_weights<kHid, kHid>(net->W3, w3);
  lane_weights<kHid, kPredOut>(net->W4, w4);
  const int on = static_cast<int>(threadIdx.x) >> 3;
  const float b1 = (on < kHid) ? net->b1[on] : 0.0f, b2 = (on < kHid) ? net->b2[on] : 0.0f;
  const float b3 = (on < kHid) ? net->b3[on] : 0.0f, b4 = (on < kPredOut) ? net->b4[on] : 0.0f;
  const double isc = (threadIdx.x < kPredIn) ? net->inv_in_scale[threadIdx.x % kPredFeat] : 0.0;
  if (threadIdx.x == 0) {
    double* row = sp->row;
    row[0] = L->Qconv;
    row[1] = __dsub_rn(L->phi0, L->phi0_prev);
    row[2] = __dsub_rn(L->Qsurf, L->Qsurf_prev);
    row[3] = L->emitted;
    row[4] = L->ion_eV;
    double err = L->err_avg, Ja = L->J_avg;
    long long ne = L->n_eval;
    if (L->had_pred) {  // running averages with weight 1/16 (a power of two: exact scaling)
      const double J = __dsub_rn(__dmul_rn(C, __dsub_rn(L->phi0, L->phi0_prev)), __dsub_rn(L->Qn, L->Q1));
      err = __dadd_rn(err, __dmul_rn(__dsub_rn(fabs(__dsub_rn(J, L->J_pred)), err), kPredAvg));
      Ja = __dadd_rn(Ja, __dmul_rn(__dsub_rn(fabs(J), Ja), kPredAvg));
      ne += 1;
      S->err_avg = err;
      S->J_avg = Ja;
      S->n_eval = ne;
    }
    for (int f = 0; f < kPredFeat; ++f) S->feat[L->pos][f] = row[f];
    S->feat_pos = (L->pos + 1) & (kPredWindow - 1);
    const int nf = min(L->n_feat + 1, kPredWindow);
    S->n_feat = nf;
    sp->full = (nf == kPredWindow);
    sp->usable = (ne >= kPredMinEval) && (err <= net->bound * Ja);
  }
  __syncthreads();
  if (!sp->full) {
    if (threadIdx.x == 0) {
      S->pred_ready = 0;
      S->J_eff = 0.0;
    }
    return;
  }
  if (threadIdx.x < kPredIn) {  // window position j (0 = oldest), feature f
    const int j = threadIdx.x / kPredFeat, f = threadIdx.x % kPredFeat;
    const double v = (j == kPredWindow - 1) ? sp->row[f] : v_old;
    sp->x[threadIdx.x] = static_cast<float>(v * isc);
  }
  __syncthreads();
  dense_lane<kPredIn, kHid, true>(w1, b1, sp->x, sp->h1);
  __syncthreads();
  dense_lane<kHid, kHid, true>(w2, b2, sp->h1, sp->h2);
  __syncthreads();
  dense_lane<kHid, kHid, true>(w3, b3, sp->h2, sp->h3);
  __syncthreads();
  dense_lane<kHid, kPredOut, false>(w4, b4, sp->h3, sp->y);
  __syncthreads();
  if (threadIdx.x == 0) {
    const double Jp = static_cast<double>(net->out_scale[1]) * static_cast<double>(sp->y[1]);
    S->J_pred = Jp;
    S->pred_ready = 1;
    S->J_eff = sp->usable ? Jp : 0.0;
  }
}
}  // namespace cpk
