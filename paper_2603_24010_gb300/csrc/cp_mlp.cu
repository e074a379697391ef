// cp_mlp.cu -- the weak-coupling predictor network: packing of an installed
// network, training samples from the diagnostics history, and the training
// kernels (initialisation, scales, forward, loss + gradient, Adam).
//
// The network (40 -> 64 -> 64 -> 64 -> 2, GELU) is far too narrow for the
// tensor cores to pay: one training step over 8192 samples is 0.1 GFLOP.
// The batch kernel therefore runs on the FP32 pipes with every weight of
// the network resident in shared memory (row-major for the backward pass,
// transposed for the forward pass, so that both read consecutive words per
// warp), 32 samples per tile, and per-CTA gradient sums kept in registers;
// a second kernel adds the per-CTA partial sums in a fixed order, so the
// gradient is bit-reproducible.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "cp_mlp.cuh"

namespace cpk {

// Parameter offsets in the FP32 master array (W[out][in] row-major).
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHid * kPredIn;  // 2560
constexpr int kOffW2 = kOffB1 + kHid;            // 2624
constexpr int kOffB2 = kOffW2 + kHid * kHid;     // 6720
constexpr int kOffW3 = kOffB2 + kHid;            // 6784
constexpr int kOffB3 = kOffW3 + kHid * kHid;     // 10880
constexpr int kOffW4 = kOffB3 + kHid;            // 10944
constexpr int kOffB4 = kOffW4 + kPredOut * kHid; // 11072
constexpr int kNParam = kOffB4 + kPredOut;       // 11074
static_assert(kNParam == CP_MLP_NPARAM, "parameter layout");
constexpr int kNWeights = kHid * kPredIn + 2 * kHid * kHid + kPredOut * kHid;  // 11072

constexpr int kTrainThreads = 256;
constexpr int kTileS = 32;         // samples per tile
constexpr int kTrainMaxCtas = 256; // rows of the partial-sum scratch
constexpr int kWorkRow = kNParam + 1;  // per-CTA gradient + loss

__device__ __forceinline__ float bf16_round(float w) {
  return __bfloat162float(__float2bfloat16_rn(w));
}
__device__ __forceinline__ uint16_t bf16_bits(float w) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(w));
}

// ---------------------------------------------------------------------------
// Installed network: BF16 weight bits and FP32 biases.
// ---------------------------------------------------------------------------
__global__ void k_pack_predictor(const float* __restrict__ p, PredNet* net) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNParam; i += gridDim.x * blockDim.x) {
    const float w = p[i];
    if (i < kOffB1) net->W1[i - kOffW1] = bf16_bits(w);
    else if (i < kOffW2) net->b1[i - kOffB1] = w;
    else if (i < kOffB2) net->W2[i - kOffW2] = bf16_bits(w);
    else if (i < kOffW3) net->b2[i - kOffB2] = w;
    else if (i < kOffB3) net->W3[i - kOffW3] = bf16_bits(w);
    else if (i < kOffW4) net->b3[i - kOffB3] = w;
    else if (i < kOffB4) net->W4[i - kOffW4] = bf16_bits(w);
    else net->b4[i - kOffB4] = w;
  }
}

// ---------------------------------------------------------------------------
// Training samples from the history rows (one thread per sample).
// ---------------------------------------------------------------------------
__global__ void k_samples(const DevParams* __restrict__ P, const cp_diag* __restrict__ h,
                          int64_t first, int64_t n, float* __restrict__ X, float* __restrict__ Y) {
  const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int64_t L = first + k;  // newest level of the window
  float* x = X + k * kPredIn;
  for (int j = 0; j < kPredWindow; ++j) {
    const int64_t m = L - (kPredWindow - 1) + j;
    const cp_diag& r = h[m];
    const cp_diag& q = h[m - 1];
    x[j * kPredFeat + 0] = static_cast<float>(r.Q_conv);
    x[j * kPredFeat + 1] = static_cast<float>(r.V_gap - q.V_gap);
    x[j * kPredFeat + 2] = static_cast<float>(r.Q_surf - q.Q_surf);
    x[j * kPredFeat + 3] = static_cast<float>(static_cast<double>(r.emitted[0]));
    x[j * kPredFeat + 4] = static_cast<float>(r.ion_energy_eV);
  }
  const cp_diag& a = h[L + 1];
  const cp_diag& b = h[L];
  const double J = P->C * (a.V_gap - b.V_gap) - (a.Q_circ - b.Q_circ);
  Y[2 * k + 0] = static_cast<float>(a.Q_conv);
  Y[2 * k + 1] = static_cast<float>(J);
}

// ---------------------------------------------------------------------------
// Initialisation: He-uniform weights from Philox draws, zero biases.
// ---------------------------------------------------------------------------
__global__ void k_mlp_init(float* __restrict__ p, uint64_t seed) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNParam; i += gridDim.x * blockDim.x) {
    int fan_in = 0;
    if (i < kOffB1) fan_in = kPredIn;
    else if (i >= kOffW2 && i < kOffB2) fan_in = kHid;
    else if (i >= kOffW3 && i < kOffB3) fan_in = kHid;
    else if (i >= kOffW4 && i < kOffB4) fan_in = kHid;
    if (fan_in == 0) {
      p[i] = 0.0f;
      continue;
    }
    const U64x4 r = philox4x64_10(static_cast<uint64_t>(i), 0, 0, 0, seed, kTagInit);
    const double u = u01(r.w[0]);
    p[i] = static_cast<float>((2.0 * u - 1.0) * sqrt(6.0 / fan_in));
  }
}

// ---------------------------------------------------------------------------
// Scales: root mean squares of the five features and two targets (one
// block, fixed summation order).
// ---------------------------------------------------------------------------
__device__ double g_scale_sums[kPredFeat + kPredOut];

__global__ void __launch_bounds__(1024) k_mlp_scales(const float* __restrict__ X,
                                                     const float* __restrict__ Y, int64_t n) {
  __shared__ double part[kPredFeat + kPredOut][32];
  double acc[kPredFeat + kPredOut];
  for (int f = 0; f < kPredFeat + kPredOut; ++f) acc[f] = 0.0;
  for (int64_t i = threadIdx.x; i < n * kPredIn; i += blockDim.x) {
    const double v = X[i];
    acc[(i % kPredIn) % kPredFeat] += v * v;
  }
  for (int64_t i = threadIdx.x; i < n * kPredOut; i += blockDim.x) {
    const double v = Y[i];
    acc[kPredFeat + (i % kPredOut)] += v * v;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int f = 0; f < kPredFeat + kPredOut; ++f) {
    double v = acc[f];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) part[f][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < kPredFeat + kPredOut) {
    double t = 0.0;
    for (int q = 0; q < static_cast<int>(blockDim.x >> 5); ++q) t += part[threadIdx.x][q];
    g_scale_sums[threadIdx.x] = t;
  }
}

__global__ void k_mlp_normalize(const float* __restrict__ X, const float* __restrict__ Y, int64_t n,
                                float s0, float s1, float s2, float s3, float s4, float o0, float o1,
                                float* __restrict__ Xn, float* __restrict__ Yn) {
  const float sx[kPredFeat] = {s0, s1, s2, s3, s4};
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n * kPredIn;
       i += stride)
    Xn[i] = X[i] / sx[(i % kPredIn) % kPredFeat];
  if (Y && Yn)
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n * kPredOut;
         i += stride)
      Yn[i] = Y[i] / ((i % kPredOut) ? o1 : o0);
}

// ---------------------------------------------------------------------------
// Batch forward (and backward) over tiles of 32 samples.
// ---------------------------------------------------------------------------
struct TrainSmem {
  float Wr[kNWeights];  // row-major W1 | W2 | W3 | W4 (BF16-rounded)
  float Wt[kNWeights];  // transposed: W1t[40][64] | W2t | W3t | W4t[64][2]
  float b[kHid * 3 + kPredOut];
  float a0[kTileS][kPredIn];
  float a1[kTileS][kHid], a2[kTileS][kHid], a3[kTileS][kHid];
  float g1[kTileS][kHid], g2[kTileS][kHid], g3[kTileS][kHid];  // GELU' then deltas
  float d4[kTileS][kPredOut];
};

constexpr int kRW1 = 0, kRW2 = kHid * kPredIn, kRW3 = kRW2 + kHid * kHid, kRW4 = kRW3 + kHid * kHid;

size_t train_smem_bytes() { return sizeof(TrainSmem); }

// one hidden layer, forward: z[s][o] = b[o] + sum_k Wt[k][o] a[s][k]
template <int IN, bool BACKWARD>
__device__ __forceinline__ void fwd_hidden(const float* Wt, const float* b, const float (*a)[IN > 0 ? IN : 1],
                                           float (*out)[kHid], float (*g)[kHid]) {
  const int o = threadIdx.x % kHid;
  const int s0 = threadIdx.x / kHid;  // 0..3
#pragma unroll
  for (int i = 0; i < kTileS / 4; ++i) {
    const int s = s0 + 4 * i;
    float z = b[o];
#pragma unroll 8
    for (int k = 0; k < IN; ++k) z = fmaf(Wt[k * kHid + o], a[s][k], z);
    out[s][o] = gelu(z);
    if (BACKWARD) g[s][o] = gelu_grad(z);
  }
}

template <bool BACKWARD>
__global__ void __launch_bounds__(kTrainThreads, 1)
k_mlp_batch(const float* __restrict__ p, const float* __restrict__ Xn, const float* __restrict__ Yn,
            int64_t n, float* __restrict__ Yhat, float* __restrict__ work) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& sm = *reinterpret_cast<TrainSmem*>(smem_raw);
  const int t = threadIdx.x;
  // weights: BF16-rounded, row-major and transposed
  for (int i = t; i < kNWeights; i += kTrainThreads) {
    int src, ti;
    if (i < kRW2) {
      src = kOffW1 + i;
      const int o = i / kPredIn, k = i % kPredIn;
      ti = k * kHid + o;
    } else if (i < kRW3) {
      src = kOffW2 + (i - kRW2);
      const int o = (i - kRW2) / kHid, k = (i - kRW2) % kHid;
      ti = kRW2 + k * kHid + o;
    } else if (i < kRW4) {
      src = kOffW3 + (i - kRW3);
      const int o = (i - kRW3) / kHid, k = (i - kRW3) % kHid;
      ti = kRW3 + k * kHid + o;
    } else {
      src = kOffW4 + (i - kRW4);
      const int o = (i - kRW4) / kHid, k = (i - kRW4) % kHid;
      ti = kRW4 + k * kPredOut + o;
    }
    const float w = bf16_round(p[src]);
    sm.Wr[i] = w;
    sm.Wt[ti] = w;
  }
  for (int i = t; i < kHid * 3 + kPredOut; i += kTrainThreads) {
    const int src = (i < kHid) ? kOffB1 + i
                    : (i < 2 * kHid) ? kOffB2 + (i - kHid)
                    : (i < 3 * kHid) ? kOffB3 + (i - 2 * kHid)
                                     : kOffB4 + (i - 3 * kHid);
    sm.b[i] = p[src];
  }
  // per-thread gradient sums (entries e = t + 256 i of each weight matrix)
  constexpr int nW1 = kHid * kPredIn / kTrainThreads;  // 10
  constexpr int nW2 = kHid * kHid / kTrainThreads;     // 16
  float gW1[nW1], gW2[nW2], gW3[nW2];
  float gW4 = 0.0f, gb = 0.0f, loss = 0.0f;
#pragma unroll
  for (int i = 0; i < nW1; ++i) gW1[i] = 0.0f;
#pragma unroll
  for (int i = 0; i < nW2; ++i) gW2[i] = gW3[i] = 0.0f;
  __syncthreads();

  const float inv_n = 1.0f / static_cast<float>(n);
  for (int64_t tile = blockIdx.x; tile * kTileS < n; tile += gridDim.x) {
    const int64_t s_base = tile * kTileS;
    const int64_t rem = n - s_base;
    const int ns = rem < kTileS ? static_cast<int>(rem) : kTileS;
    for (int i = t; i < kTileS * kPredIn; i += kTrainThreads) {
      const int s = i / kPredIn, k = i % kPredIn;
      sm.a0[s][k] = (s < ns) ? Xn[(s_base + s) * kPredIn + k] : 0.0f;
    }
    __syncthreads();
    fwd_hidden<kPredIn, BACKWARD>(sm.Wt + kRW1, sm.b, sm.a0, sm.a1, sm.g1);
    __syncthreads();
    fwd_hidden<kHid, BACKWARD>(sm.Wt + kRW2, sm.b + kHid, sm.a1, sm.a2, sm.g2);
    __syncthreads();
    fwd_hidden<kHid, BACKWARD>(sm.Wt + kRW3, sm.b + 2 * kHid, sm.a2, sm.a3, sm.g3);
    __syncthreads();
    if (t < kTileS * kPredOut) {  // output layer, linear
      const int o = t & 1, s = t >> 1;
      float z = sm.b[3 * kHid + o];
#pragma unroll 8
      for (int k = 0; k < kHid; ++k) z = fmaf(sm.Wt[kRW4 + k * kPredOut + o], sm.a3[s][k], z);
      if (!BACKWARD) {
        if (s < ns) Yhat[(s_base + s) * kPredOut + o] = z;
      } else {
        float d = 0.0f;
        if (s < ns) {
          const float e = z - Yn[(s_base + s) * kPredOut + o];
          d = e * inv_n;
          loss = fmaf(0.5f * e, e * inv_n, loss);
        }
        sm.d4[s][o] = d;
      }
    }
    if (!BACKWARD) {
      __syncthreads();
      continue;
    }
    __syncthreads();
    // delta of layer 3 (in place over its GELU'), gradient of layer 4
    {
      const int k = t % kHid, s0 = t / kHid;
#pragma unroll
      for (int i = 0; i < kTileS / 4; ++i) {
        const int s = s0 + 4 * i;
        const float back = sm.Wr[kRW4 + k] * sm.d4[s][0] + sm.Wr[kRW4 + kHid + k] * sm.d4[s][1];
        sm.g3[s][k] *= back;
      }
      if (t < kPredOut * kHid) {
        const int o = t / kHid;
        float acc = 0.0f;
        for (int s = 0; s < kTileS; ++s) acc = fmaf(sm.d4[s][o], sm.a3[s][k], acc);
        gW4 += acc;
      }
    }
    __syncthreads();
    // delta of layer 2, gradient of layer 3 (W3: d3 x a2)
    {
      const int k = t % kHid, s0 = t / kHid;
#pragma unroll
      for (int i = 0; i < kTileS / 4; ++i) {
        const int s = s0 + 4 * i;
        float back = 0.0f;
#pragma unroll 8
        for (int o = 0; o < kHid; ++o) back = fmaf(sm.Wr[kRW3 + o * kHid + k], sm.g3[s][o], back);
        sm.g2[s][k] *= back;
      }
#pragma unroll
      for (int i = 0; i < nW2; ++i) {
        const int o = s0 + 4 * i;
        float acc = 0.0f;
        for (int s = 0; s < kTileS; ++s) acc = fmaf(sm.g3[s][o], sm.a2[s][k], acc);
        gW3[i] += acc;
      }
    }
    __syncthreads();
    // delta of layer 1, gradient of layer 2 (W2: d2 x a1)
    {
      const int k = t % kHid, s0 = t / kHid;
#pragma unroll
      for (int i = 0; i < kTileS / 4; ++i) {
        const int s = s0 + 4 * i;
        float back = 0.0f;
#pragma unroll 8
        for (int o = 0; o < kHid; ++o) back = fmaf(sm.Wr[kRW2 + o * kHid + k], sm.g2[s][o], back);
        sm.g1[s][k] *= back;
      }
#pragma unroll
      for (int i = 0; i < nW2; ++i) {
        const int o = s0 + 4 * i;
        float acc = 0.0f;
        for (int s = 0; s < kTileS; ++s) acc = fmaf(sm.g2[s][o], sm.a1[s][k], acc);
        gW2[i] += acc;
      }
    }
    __syncthreads();
    // gradient of layer 1 (W1: d1 x a0) and of the biases
#pragma unroll
    for (int i = 0; i < nW1; ++i) {
      const int e = t + kTrainThreads * i;
      const int o = e / kPredIn, k = e % kPredIn;
      float acc = 0.0f;
      for (int s = 0; s < kTileS; ++s) acc = fmaf(sm.g1[s][o], sm.a0[s][k], acc);
      gW1[i] += acc;
    }
    if (t < 3 * kHid + kPredOut) {
      float acc = 0.0f;
      if (t < kHid) for (int s = 0; s < kTileS; ++s) acc += sm.g1[s][t];
      else if (t < 2 * kHid) for (int s = 0; s < kTileS; ++s) acc += sm.g2[s][t - kHid];
      else if (t < 3 * kHid) for (int s = 0; s < kTileS; ++s) acc += sm.g3[s][t - 2 * kHid];
      else for (int s = 0; s < kTileS; ++s) acc += sm.d4[s][t - 3 * kHid];
      gb += acc;
    }
    __syncthreads();
  }
  if (!BACKWARD) return;
  // this CTA's partial sums, in parameter order
  float* w = work + static_cast<int64_t>(blockIdx.x) * kWorkRow;
#pragma unroll
  for (int i = 0; i < nW1; ++i) w[kOffW1 + t + kTrainThreads * i] = gW1[i];
  {
    const int k = t % kHid, s0 = t / kHid;
#pragma unroll
    for (int i = 0; i < nW2; ++i) {
      w[kOffW2 + (s0 + 4 * i) * kHid + k] = gW2[i];
      w[kOffW3 + (s0 + 4 * i) * kHid + k] = gW3[i];
    }
  }
  if (t < kPredOut * kHid) w[kOffW4 + t] = gW4;
  if (t < kHid) w[kOffB1 + t] = gb;
  else if (t < 2 * kHid) w[kOffB2 + t - kHid] = gb;
  else if (t < 3 * kHid) w[kOffB3 + t - 2 * kHid] = gb;
  else if (t < 3 * kHid + kPredOut) w[kOffB4 + t - 3 * kHid] = gb;
  // loss: block sum in a fixed order
  __shared__ float lpart[kTrainThreads / 32];
  float l = loss;
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((t & 31) == 0) lpart[t >> 5] = l;
  __syncthreads();
  if (t == 0) {
    float s = 0.0f;
    for (int q = 0; q < kTrainThreads / 32; ++q) s += lpart[q];
    w[kNParam] = s;
  }
}

__global__ void k_mlp_reduce(const float* __restrict__ work, int ctas, float* __restrict__ grad,
                             float* __restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kWorkRow) return;
  float s = 0.0f;
  for (int b = 0; b < ctas; ++b) s += work[static_cast<int64_t>(b) * kWorkRow + i];
  if (i < kNParam) grad[i] = s;
  else *loss = s;
}

__global__ void k_mlp_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, float lr, float b1, float b2, float eps, float c1,
                           float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNParam) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// ---------------------------------------------------------------------------
// Host-side launchers
// ---------------------------------------------------------------------------
cudaError_t pack_predictor_launch(const float* params, PredNet* net, cudaStream_t st) {
  k_pack_predictor<<<(kNParam + 255) / 256, 256, 0, st>>>(params, net);
  return cudaGetLastError();
}

cudaError_t samples_launch(const DevParams* P, const cp_diag* hist, int64_t first, int64_t n,
                           float* X, float* Y, cudaStream_t st) {
  const int64_t blocks = (n + 127) / 128;
  k_samples<<<static_cast<unsigned>(blocks), 128, 0, st>>>(P, hist, first, n, X, Y);
  return cudaGetLastError();
}

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return sms > 0 ? sms : 1;
}

cudaError_t mlp_batch_launch(bool backward, const float* p, const float* Xn, const float* Yn,
                             int64_t n, float* Yhat, float* work, int* ctas_out, cudaStream_t st) {
  const size_t smem = sizeof(TrainSmem);
  cudaError_t e = backward
                      ? cudaFuncSetAttribute(k_mlp_batch<true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem))
                      : cudaFuncSetAttribute(k_mlp_batch<false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const int64_t tiles = (n + kTileS - 1) / kTileS;
  int ctas = static_cast<int>(std::min<int64_t>(tiles, static_cast<int64_t>(sm_count())));
  if (backward) ctas = std::min(ctas, kTrainMaxCtas);
  if (ctas < 1) ctas = 1;
  if (ctas_out) *ctas_out = ctas;
  if (backward)
    k_mlp_batch<true><<<ctas, kTrainThreads, smem, st>>>(p, Xn, Yn, n, Yhat, work);
  else
    k_mlp_batch<false><<<ctas, kTrainThreads, smem, st>>>(p, Xn, Yn, n, Yhat, work);
  return cudaGetLastError();
}

}  // namespace cpk

// ---------------------------------------------------------------------------
// C ABI of the training kernels
// ---------------------------------------------------------------------------
namespace {
cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }
int rc_of(cudaError_t e) { return e == cudaSuccess ? CP_OK : CP_ERR_CUDA; }
}  // namespace

extern "C" {

int cp_mlp_init(float* params, uint64_t seed, void* stream) {
  if (!params) return CP_ERR_ARG;
  cpk::k_mlp_init<<<(cpk::kNParam + 255) / 256, 256, 0, as_stream(stream)>>>(params, seed);
  return rc_of(cudaGetLastError());
}

int cp_mlp_scales(const float* X, const float* Y, int64_t n, cp_predictor* norm, void* stream) {
  if (!X || !Y || !norm || n <= 0) return CP_ERR_ARG;
  cudaStream_t st = as_stream(stream);
  cpk::k_mlp_scales<<<1, 1024, 0, st>>>(X, Y, n);
  cudaError_t e = cudaGetLastError();
  double sums[cpk::kPredFeat + cpk::kPredOut];
  if (e == cudaSuccess)
    e = cudaMemcpyFromSymbolAsync(sums, cpk::g_scale_sums, sizeof(sums), 0, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return CP_ERR_CUDA;
  for (int f = 0; f < cpk::kPredFeat; ++f) {
    const double r = std::sqrt(sums[f] / (static_cast<double>(n) * cpk::kPredWindow));
    norm->in_scale[f] = (r > 0.0 && std::isfinite(r)) ? static_cast<float>(r) : 1.0f;
  }
  for (int o = 0; o < cpk::kPredOut; ++o) {
    const double r = std::sqrt(sums[cpk::kPredFeat + o] / static_cast<double>(n));
    norm->out_scale[o] = (r > 0.0 && std::isfinite(r)) ? static_cast<float>(r) : 1.0f;
  }
  return CP_OK;
}

int cp_mlp_normalize(const float* X, const float* Y, int64_t n, const cp_predictor* norm, float* Xn,
                     float* Yn, void* stream) {
  if (!X || !Xn || !norm || n < 0 || ((Y == nullptr) != (Yn == nullptr))) return CP_ERR_ARG;
  if (n == 0) return CP_OK;
  const int64_t blocks = std::min<int64_t>((n * cpk::kPredIn + 255) / 256, 4096);
  cpk::k_mlp_normalize<<<static_cast<unsigned>(blocks), 256, 0, as_stream(stream)>>>(
      X, Y, n, norm->in_scale[0], norm->in_scale[1], norm->in_scale[2], norm->in_scale[3],
      norm->in_scale[4], norm->out_scale[0], norm->out_scale[1], Xn, Yn);
  return rc_of(cudaGetLastError());
}

int cp_mlp_forward(const float* params, const float* Xn, int64_t n, float* Yhat, void* stream) {
  if (!params || !Xn || !Yhat || n < 0) return CP_ERR_ARG;
  if (n == 0) return CP_OK;
  return rc_of(cpk::mlp_batch_launch(false, params, Xn, nullptr, n, Yhat, nullptr, nullptr,
                                     as_stream(stream)));
}

int64_t cp_mlp_work_floats(void) {
  return static_cast<int64_t>(cpk::kTrainMaxCtas) * cpk::kWorkRow;
}

int cp_mlp_loss_grad(const float* params, const float* Xn, const float* Yn, int64_t n, float* grad,
                     float* loss, float* work, void* stream) {
  if (!params || !Xn || !Yn || !grad || !loss || !work || n <= 0) return CP_ERR_ARG;
  cudaStream_t st = as_stream(stream);
  int ctas = 0;
  cudaError_t e = cpk::mlp_batch_launch(true, params, Xn, Yn, n, nullptr, work, &ctas, st);
  if (e != cudaSuccess) return CP_ERR_CUDA;
  cpk::k_mlp_reduce<<<(cpk::kWorkRow + 255) / 256, 256, 0, st>>>(work, ctas, grad, loss);
  return rc_of(cudaGetLastError());
}

int cp_mlp_adam(float* params, const float* grad, float* m, float* v, int64_t t, float lr,
                float beta1, float beta2, float eps, void* stream) {
  if (!params || !grad || !m || !v || t < 1 || !(lr > 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
      !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
    return CP_ERR_ARG;
  const double c1 = 1.0 / (1.0 - std::pow(static_cast<double>(beta1), static_cast<double>(t)));
  const double c2 = 1.0 / (1.0 - std::pow(static_cast<double>(beta2), static_cast<double>(t)));
  cpk::k_mlp_adam<<<(cpk::kNParam + 255) / 256, 256, 0, as_stream(stream)>>>(
      params, grad, m, v, lr, beta1, beta2, eps, static_cast<float>(c1), static_cast<float>(c2));
  return rc_of(cudaGetLastError());
}

}  // extern "C"
