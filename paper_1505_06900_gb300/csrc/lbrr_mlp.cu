// Tensor-core kernels of the learned closure's network (BF16 operands, FP32
// accumulation): y = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3, x in R^288,
// hidden 64 + 64, y in R^32 (17 outputs used), with the loss
// mean((y - t)^2) over the used outputs, its backward pass and Adam.
//
// mlp_train_kernel is persistent: each block walks 64-row tiles of the batch
// (the forward pass alone runs on the tcgen05 kernels of lbrr_mlp_tc.cu).
// A warp owns 16 rows. Layer 1 takes its A fragments from the staged input
// tile (ldmatrix) and its B fragments straight from the K-major BF16 weights;
// every later layer takes the previous layer's accumulators, passed through
// bias + tanh and rounded to BF16, as its A fragments without leaving
// registers (the m16n8 accumulator layout is the m16k16 operand layout of the
// next product). The backward data pass runs the same way on W3^T and W2^T
// copies. For the weight gradients the block stages the BF16 tiles of x, h1,
// h2, dh1, dh2 and dy in shared memory and multiplies their transposes
// (ldmatrix .trans) into FP32 accumulators in shared memory, one owner warp
// per output tile; at the end each block writes its partial sums, which
// mlp_reduce_adam_kernel adds in block order (deterministic) before the Adam
// update and the refresh of the BF16 weight copies.
#include <cstdint>

#include "lbrr_launch.h"
#include "lbrr_mlp.h"
#include "lbrr_mma.cuh"

namespace lbrr {

namespace {

constexpr int kRows = 64;      // rows per tile (4 warps x 16)
constexpr int kThreads = 128;  // 4 warps
constexpr int kXs = kMlpIn + 8;    // smem row strides (elements), chosen so that
constexpr int kHs = kMlpHidden + 8;  // eight 16-byte rows hit eight distinct
constexpr int kYs = kMlpOut + 8;     // 16-byte bank groups (ldmatrix without conflicts)

struct TrainSmem {
  __nv_bfloat16 x[kRows][kXs];
  __nv_bfloat16 h1[kRows][kHs], h2[kRows][kHs], dh1[kRows][kHs], dh2[kRows][kHs];
  __nv_bfloat16 dy[kRows][kYs];
  float gw1[kMlpHidden][kMlpIn];
  float gw2[kMlpHidden][kMlpHidden];
  float gw3[kMlpOut][kMlpHidden];
  float gb_warp[4][kMlpHidden + kMlpHidden + kMlpOut];  // per-warp bias-gradient sums
  float gb[kMlpHidden + kMlpHidden + kMlpOut];
  float loss[4];
};

// Store accumulator tiles (16 rows of a warp) as BF16 into a smem tile.
template <int NT, int LD>
__device__ __forceinline__ void store_tile(__nv_bfloat16 (*s)[LD], int r0, int g, int t,
                                           const float (&acc)[NT][4]) {
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    *reinterpret_cast<uint32_t *>(&s[r0 + g][8 * nt + 2 * t]) = pack_bf16(acc[nt][0], acc[nt][1]);
    *reinterpret_cast<uint32_t *>(&s[r0 + g + 8][8 * nt + 2 * t]) =
        pack_bf16(acc[nt][2], acc[nt][3]);
  }
}

// Column sums over the warp's 16 rows of NT accumulator tiles, into dst[8 nt + c].
template <int NT>
__device__ __forceinline__ void col_sums(const float (&acc)[NT][4], int g, int t, float *dst) {
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    float s0 = acc[nt][0] + acc[nt][2], s1 = acc[nt][1] + acc[nt][3];
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if (g == 0) {
      dst[8 * nt + 2 * t] = s0;
      dst[8 * nt + 2 * t + 1] = s1;
    }
  }
}

// acc[m-tile rows j0.., n-tiles] += sum over the tile's 64 rows of
// Ls[m][j0 + .]^T * Rs[m][n0 + .]; NP pairs of n8 tiles starting at column n0.
template <int LDL, int LDR, int NP>
__device__ __forceinline__ void wgrad(const __nv_bfloat16 (*Ls)[LDL], int j0,
                                      const __nv_bfloat16 (*Rs)[LDR], int n0, int lane,
                                      float *out, int ldo) {
  const int g = lane >> 2, t = lane & 3, i = lane >> 3, r = lane & 7;
  uint32_t a[4][4];
#pragma unroll
  for (int ks = 0; ks < 4; ++ks)  // A(j, m) = Ls[m][j]: transposed 8x8 blocks
    ldsm_x4_t(a[ks], &Ls[16 * ks + 8 * (i >> 1) + r][j0 + 8 * (i & 1)]);
#pragma unroll 2
  for (int p = 0; p < NP; ++p) {
    float d0[4] = {0.f, 0.f, 0.f, 0.f}, d1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      uint32_t b[4];  // B(m, n) = Rs[m][n]: two n8 tiles
      ldsm_x4_t(b, &Rs[16 * ks + 8 * (i & 1) + r][n0 + 16 * p + 8 * (i >> 1)]);
      mma16816(d0, a[ks], b[0], b[1]);
      mma16816(d1, a[ks], b[2], b[3]);
    }
    float *o0 = out + (long long)(j0 + g) * ldo + n0 + 16 * p + 2 * t;
    float *o1 = o0 + 8 * ldo;
    o0[0] += d0[0];
    o0[1] += d0[1];
    o1[0] += d0[2];
    o1[1] += d0[3];
    o0[8] += d1[0];
    o0[9] += d1[1];
    o1[8] += d1[2];
    o1[9] += d1[3];
  }
}

// Trace rows (TRACE instantiation): FP32 values of row r at trace[r][c] for
// the columns col0 + 8 nt + 2 t (+1) of NT accumulator tiles.
template <int NT>
__device__ __forceinline__ void trace_tile(float *__restrict__ trace, long long ra, long long rb,
                                           long long M, int col0, int t,
                                           const float (&acc)[NT][4]) {
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    const int c = col0 + 8 * nt + 2 * t;
    if (ra < M)
      *reinterpret_cast<float2 *>(trace + ra * kMlpTrace + c) = make_float2(acc[nt][0], acc[nt][1]);
    if (rb < M)
      *reinterpret_cast<float2 *>(trace + rb * kMlpTrace + c) = make_float2(acc[nt][2], acc[nt][3]);
  }
}

template <bool TRACE = false>
__global__ void __launch_bounds__(kThreads)
    mlp_train_kernel(MlpDevice p, const __nv_bfloat16 *__restrict__ X,
                     const float *__restrict__ T, long long M, float *__restrict__ gpart,
                     float *__restrict__ lpart, float *__restrict__ trace) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem &s = *reinterpret_cast<TrainSmem *>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int r0 = 16 * warp;
  const long long ntiles = (M + kRows - 1) / kRows;
  const float inv_n = 1.0f / ((float)M * (float)kMlpOutUsed);

  for (int k = tid; k < kMlpHidden * kMlpIn; k += kThreads) (&s.gw1[0][0])[k] = 0.f;
  for (int k = tid; k < kMlpHidden * kMlpHidden; k += kThreads) (&s.gw2[0][0])[k] = 0.f;
  for (int k = tid; k < kMlpOut * kMlpHidden; k += kThreads) (&s.gw3[0][0])[k] = 0.f;
  for (int k = tid; k < 2 * kMlpHidden + kMlpOut; k += kThreads) s.gb[k] = 0.f;
  float loss_acc = 0.f;

  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long row0 = tile * kRows;
    // ---- stage the input rows (rows past M are zero)
    for (int c = tid; c < kRows * (kMlpIn / 8); c += kThreads) {
      const int r = c / (kMlpIn / 8), k = c - r * (kMlpIn / 8);
      if (row0 + r < M)
        cp_async16(&s.x[r][8 * k], X + (row0 + r) * kMlpIn + 8 * k);
      else
        *reinterpret_cast<uint4 *>(&s.x[r][8 * k]) = make_uint4(0, 0, 0, 0);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();

    // ---- layer 1: [16 x 288] x [288 x 64]
    float h1[8][4] = {};
#pragma unroll 2
    for (int ks = 0; ks < kMlpIn / 16; ++ks) {
      uint32_t a[4];
      ldsm_x4(a, &s.x[r0 + (lane & 15)][16 * ks + 8 * (lane >> 4)]);
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        uint32_t b0, b1;
        b_frag(b0, b1, p.w1, kMlpIn, 8 * nt, 16 * ks, g, t);
        mma16816(h1[nt], a, b0, b1);
      }
    }
    uint32_t a1[4][4];
    act_to_frags<8>(h1, p.b1, t, a1);
    const long long ra = row0 + r0 + g, rb = ra + 8;
    if (TRACE) trace_tile<8>(trace, ra, rb, M, kTraceH1, t, h1);
    // ---- layer 2
    float h2[8][4] = {};
#pragma unroll
    for (int ks = 0; ks < 4; ++ks)
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        uint32_t b0, b1;
        b_frag(b0, b1, p.w2, kMlpHidden, 8 * nt, 16 * ks, g, t);
        mma16816(h2[nt], a1[ks], b0, b1);
      }
    uint32_t a2[4][4];
    act_to_frags<8>(h2, p.b2, t, a2);
    if (TRACE) trace_tile<8>(trace, ra, rb, M, kTraceH2, t, h2);
    // ---- layer 3
    float y[4][4] = {};
#pragma unroll
    for (int ks = 0; ks < 4; ++ks)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        uint32_t b0, b1;
        b_frag(b0, b1, p.w3, kMlpHidden, 8 * nt, 16 * ks, g, t);
        mma16816(y[nt], a2[ks], b0, b1);
      }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int c = 8 * nt + 2 * t;
      y[nt][0] += p.b3[c];
      y[nt][1] += p.b3[c + 1];
      y[nt][2] += p.b3[c];
      y[nt][3] += p.b3[c + 1];
    }
    if (TRACE) trace_tile<4>(trace, ra, rb, M, kTraceY, t, y);

    // ---- loss and dy = 2 (y - t) / (M * 17) on the used outputs of valid rows
    float dy[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const long long r = e < 2 ? ra : rb;
        const int c = 8 * nt + 2 * t + (e & 1);
        float d = 0.f;
        if (r < M && c < kMlpOutUsed) d = y[nt][e] - T[r * kMlpOut + c];
        loss_acc += d * d;
        dy[nt][e] = 2.0f * d * inv_n;
      }
    }
    if (TRACE) trace_tile<4>(trace, ra, rb, M, kTraceDy, t, dy);
    uint32_t ady[2][4];
    to_frags<4>(dy, ady);
    // ---- dh2 = (dy W3) * (1 - h2^2), with W3^T [64][32] K-major
    float g2[8][4] = {};
#pragma unroll
    for (int ks = 0; ks < 2; ++ks)
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        uint32_t b0, b1;
        b_frag(b0, b1, p.w3t, kMlpOut, 8 * nt, 16 * ks, g, t);
        mma16816(g2[nt], ady[ks], b0, b1);
      }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) g2[nt][e] *= 1.0f - h2[nt][e] * h2[nt][e];
    if (TRACE) trace_tile<8>(trace, ra, rb, M, kTraceDh2, t, g2);
    uint32_t ag2[4][4];
    to_frags<8>(g2, ag2);
    // ---- dh1 = (dh2 W2) * (1 - h1^2), with W2^T [64][64]
    float g1[8][4] = {};
#pragma unroll
    for (int ks = 0; ks < 4; ++ks)
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        uint32_t b0, b1;
        b_frag(b0, b1, p.w2t, kMlpHidden, 8 * nt, 16 * ks, g, t);
        mma16816(g1[nt], ag2[ks], b0, b1);
      }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) g1[nt][e] *= 1.0f - h1[nt][e] * h1[nt][e];
    if (TRACE) trace_tile<8>(trace, ra, rb, M, kTraceDh1, t, g1);

    // ---- stage the BF16 tiles for the weight gradients, bias gradients per warp
    store_tile<8, kHs>(s.h1, r0, g, t, h1);
    store_tile<8, kHs>(s.h2, r0, g, t, h2);
    store_tile<8, kHs>(s.dh1, r0, g, t, g1);
    store_tile<8, kHs>(s.dh2, r0, g, t, g2);
    store_tile<4, kYs>(s.dy, r0, g, t, dy);
    col_sums<8>(g1, g, t, &s.gb_warp[warp][0]);
    col_sums<8>(g2, g, t, &s.gb_warp[warp][kMlpHidden]);
    col_sums<4>(dy, g, t, &s.gb_warp[warp][2 * kMlpHidden]);
    __syncthreads();

    // ---- weight gradients of this tile into the block's FP32 accumulators
    // dW1 [64 x 288] = dh1^T x : warp w owns rows 16w..16w+15
    wgrad<kHs, kXs, kMlpIn / 16>(s.dh1, 16 * warp, s.x, 0, lane, &s.gw1[0][0], kMlpIn);
    // dW2 [64 x 64] = dh2^T h1
    wgrad<kHs, kHs, kMlpHidden / 16>(s.dh2, 16 * warp, s.h1, 0, lane, &s.gw2[0][0], kMlpHidden);
    // dW3 [32 x 64] = dy^T h2 : warp w owns rows 16 (w % 2).., columns 32 (w / 2)..
    wgrad<kYs, kHs, 2>(s.dy, 16 * (warp & 1), s.h2, 32 * (warp >> 1), lane, &s.gw3[0][0],
                       kMlpHidden);
    for (int k = tid; k < 2 * kMlpHidden + kMlpOut; k += kThreads)
      s.gb[k] += ((s.gb_warp[0][k] + s.gb_warp[1][k]) + s.gb_warp[2][k]) + s.gb_warp[3][k];
    __syncthreads();
  }

  // ---- block partials in the packed parameter order
  float *o = gpart + (long long)blockIdx.x * kMlpParams;
  for (int k = tid; k < kMlpHidden * kMlpIn; k += kThreads) o[kOffW1 + k] = (&s.gw1[0][0])[k];
  for (int k = tid; k < kMlpHidden; k += kThreads) o[kOffB1 + k] = s.gb[k];
  for (int k = tid; k < kMlpHidden * kMlpHidden; k += kThreads) o[kOffW2 + k] = (&s.gw2[0][0])[k];
  for (int k = tid; k < kMlpHidden; k += kThreads) o[kOffB2 + k] = s.gb[kMlpHidden + k];
  for (int k = tid; k < kMlpOut * kMlpHidden; k += kThreads) o[kOffW3 + k] = (&s.gw3[0][0])[k];
  for (int k = tid; k < kMlpOut; k += kThreads) o[kOffB3 + k] = s.gb[2 * kMlpHidden + k];
  for (int off = 16; off > 0; off >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, off);
  if (lane == 0) s.loss[warp] = loss_acc;
  __syncthreads();
  if (tid == 0) lpart[blockIdx.x] = ((s.loss[0] + s.loss[1]) + s.loss[2]) + s.loss[3];
}

// Sum of the block partials (fixed order), optional Adam update of the FP32
// master parameters and refresh of the BF16 copies.
__global__ void mlp_reduce_adam_kernel(MlpDevice p, const float *__restrict__ gpart, int nparts,
                                       float *__restrict__ grad_out, int adam, float lr,
                                       float bc1, float bc2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kMlpParams) return;
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

size_t mlp_train_smem() { return sizeof(TrainSmem); }

cudaError_t launch_mlp_train(const MlpDevice &p, const void *X, const float *T, long long M,
                             float *gpart, float *lpart, int nblocks, cudaStream_t st,
                             float *trace) {
  const size_t smem = sizeof(TrainSmem);
  if (!T) return cudaErrorInvalidValue;
  auto kern = trace ? mlp_train_kernel<true> : mlp_train_kernel<false>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<nblocks, kThreads, smem, st>>>(p, static_cast<const __nv_bfloat16 *>(X), T, M, gpart,
                                       lpart, trace);
  return cudaGetLastError();
}

cudaError_t launch_mlp_reduce(const MlpDevice &p, const float *gpart, int nparts, float *grad_out,
                              int adam, float lr, float bc1, float bc2, const float *lpart,
                              double *loss_out, cudaStream_t st) {
  mlp_reduce_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(p, gpart, nparts, grad_out,
                                                                  adam, lr, bc1, bc2);
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
