// Warp-level tensor-core helpers (mma.sync m16n8k16, BF16 in, FP32
// accumulate) shared by the network kernels and the closure step.
//
// Fragment layouts (g = lane / 4, t = lane % 4):
//   A (16 x 16, row): a0 = (g, 2t..2t+1), a1 = (g+8, 2t..), a2 = (g, 2t+8..), a3 = (g+8, 2t+8..)
//   B (16 x 8, col):  b0 = (k 2t..2t+1, n g), b1 = (k 2t+8.., n g)
//   C (16 x 8):       c0, c1 = (g, 2t..2t+1), c2, c3 = (g+8, 2t..2t+1)
// so the accumulators of two adjacent n8 tiles are, once rounded to BF16, the
// A operand of one k16 step of the next product.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace lbrr {

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(s));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void *p) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(s));
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

// B fragment (k = 2t, 2t+1 and 2t+8, 2t+9; n = g) of a K-major weight W[n][k].
__device__ __forceinline__ void b_frag(uint32_t &b0, uint32_t &b1, const __nv_bfloat16 *W, int ld,
                                       int n0, int k0, int g, int t) {
  const __nv_bfloat16 *p = W + (long long)(n0 + g) * ld + k0 + 2 * t;
  b0 = __ldg(reinterpret_cast<const unsigned int *>(p));
  b1 = __ldg(reinterpret_cast<const unsigned int *>(p + 8));
}

// A fragments of the next layer from NT accumulator tiles (bias + tanh first).
// Hardware tanh (tanh.approx.f32, relative error ~2^-11, below the BF16
// rounding the activations get next); the same in training and inference.
__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int NT>
__device__ __forceinline__ void act_to_frags(float (&acc)[NT][4], const float *bias, int t,
                                             uint32_t (&a)[NT / 2][4]) {
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    const float b0 = bias[8 * nt + 2 * t], b1 = bias[8 * nt + 2 * t + 1];
    acc[nt][0] = tanh_approx(acc[nt][0] + b0);
    acc[nt][1] = tanh_approx(acc[nt][1] + b1);
    acc[nt][2] = tanh_approx(acc[nt][2] + b0);
    acc[nt][3] = tanh_approx(acc[nt][3] + b1);
  }
#pragma unroll
  for (int ks = 0; ks < NT / 2; ++ks) {
    a[ks][0] = pack_bf16(acc[2 * ks][0], acc[2 * ks][1]);
    a[ks][1] = pack_bf16(acc[2 * ks][2], acc[2 * ks][3]);
    a[ks][2] = pack_bf16(acc[2 * ks + 1][0], acc[2 * ks + 1][1]);
    a[ks][3] = pack_bf16(acc[2 * ks + 1][2], acc[2 * ks + 1][3]);
  }
}

// A fragments from plain accumulators (no activation).
template <int NT>
__device__ __forceinline__ void to_frags(const float (&acc)[NT][4], uint32_t (&a)[NT / 2][4]) {
#pragma unroll
  for (int ks = 0; ks < NT / 2; ++ks) {
    a[ks][0] = pack_bf16(acc[2 * ks][0], acc[2 * ks][1]);
    a[ks][1] = pack_bf16(acc[2 * ks][2], acc[2 * ks][3]);
    a[ks][2] = pack_bf16(acc[2 * ks + 1][0], acc[2 * ks + 1][1]);
    a[ks][3] = pack_bf16(acc[2 * ks + 1][2], acc[2 * ks + 1][3]);
  }
}


}  // namespace lbrr
