// Activation and BF16 packing helpers shared by the network kernels and the
// closure step.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace lbrr {

// two floats rounded to BF16 (nearest even), lo in the low half
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}

// Hardware tanh (tanh.approx.f32, relative error ~2^-11, below the BF16
// rounding the activations get next); the same in training and inference.
__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

}  // namespace lbrr
