// Reduction and Adam kernels of the closure network's training (the
// forward + backward pass itself is lbrr_mlp_train.cu): the block partial
// gradients are summed in block order (deterministic), then an optional Adam
// step updates the FP32 master parameters and refreshes their BF16 copies
// (K-major weights and the transposed copies of W2 and W3).
#include <cstdint>

#include "lbrr_launch.h"
#include "lbrr_mlp.h"
#include "lbrr_act.cuh"

namespace lbrr {

namespace {

// Sum of the block partials (fixed order), optional Adam update of the FP32
// master parameters and refresh of the BF16 copies; nothing when the
// training kernel recorded a timeout (its partials are incomplete).
__global__ void mlp_reduce_adam_kernel(MlpDevice p, const float *__restrict__ gpart, int nparts,
                                       float *__restrict__ grad_out, int adam, float lr,
                                       float bc1, float bc2, const int *status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kMlpParams || *status) return;
  float gsum = 0.f;
  for (int b = 0; b < nparts; ++b) gsum += gpart[(long long)b * kMlpParams + k];
  if (grad_out) grad_out[k] = gsum;
  if (!adam) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float m = b1 * p.adam_m[k] + (1.f - b1) * gsum;
  const float v = b2 * p.adam_v[k] + (1.f - b2) * gsum * gsum;
  p.adam_m[k] = m;
  p.adam_v[k] = v;
  const float w = p.params[k] - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
  p.params[k] = w;
  mlp_refresh_one(p, k, w);
}

__global__ void mlp_refresh_kernel(MlpDevice p) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < kMlpParams) mlp_refresh_one(p, k, p.params[k]);
}

__global__ void loss_sum_kernel(const float *__restrict__ lpart, int n, double *out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < n; ++b) s += lpart[b];
    *out = s;
  }
}

}  // namespace

__device__ void mlp_refresh_one(MlpDevice p, int k, float w) {
  const __nv_bfloat16 v = __float2bfloat16_rn(w);
  if (k < kOffB1) {
    p.w1[k] = v;
  } else if (k >= kOffW2 && k < kOffB2) {
    const int q = k - kOffW2, n = q / kMlpHidden, c = q % kMlpHidden;
    p.w2[q] = v;
    p.w2t[c * kMlpHidden + n] = v;
  } else if (k >= kOffW3 && k < kOffB3) {
    const int q = k - kOffW3, n = q / kMlpHidden, c = q % kMlpHidden;
    p.w3[q] = v;
    p.w3t[c * kMlpOut + n] = v;
  }
}

cudaError_t launch_mlp_reduce(const MlpDevice &p, const float *gpart, int nparts, float *grad_out,
                              int adam, float lr, float bc1, float bc2, const float *lpart,
                              double *loss_out, const int *status, cudaStream_t st) {
  mlp_reduce_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(p, gpart, nparts, grad_out,
                                                                  adam, lr, bc1, bc2, status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !loss_out) return e;
  loss_sum_kernel<<<1, 32, 0, st>>>(lpart, nparts, loss_out);
  return cudaGetLastError();
}

cudaError_t launch_mlp_refresh(const MlpDevice &p, cudaStream_t st) {
  mlp_refresh_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace lbrr
