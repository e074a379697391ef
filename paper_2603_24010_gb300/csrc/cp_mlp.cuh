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

}  // namespace cpk
