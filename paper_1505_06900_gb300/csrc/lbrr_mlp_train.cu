// Training pass of the closure network on the 5th-generation tensor cores
// (tcgen05): for a batch X [M][288] (BF16) with targets T [M][32], the
// forward pass y = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3, the loss
// sum over rows and used outputs of (y - t)^2, its gradient dy = 2 (y - t) /
// (17 M) on the used outputs, the back-propagated dh2 = (dy W3) (1 - h2^2),
// dh1 = (dh2 W2) (1 - h1^2), and every weight and bias gradient, as per-block
// partial sums that mlp_reduce_adam_kernel adds in block order.
//
// One persistent block per SM walks 128-row tiles; thread r and r + 128 own
// row r (TMEM lane r), each half of its columns. Per tile one thread issues,
// in turn: layer 1 (X W1^T), layer 2, layer 3, the two backward products
// (dy W3, dh2 W2) and the three weight-gradient products, each committed to
// one mbarrier that all threads wait on (bounded). Operands are BF16 tiles in
// shared memory in the canonical layout without swizzle (8-row x 16-byte core
// matrices); the weight gradients read the same tiles transposed, as
// MN-major operands (the transpose bits of the instruction descriptor; the
// leading byte offset is then the stride between core matrices along K, the
// batch rows, and the stride byte offset the one along M or N):
//   gW1^T [288 x 64] = X^T dh1    (three M = 128 blocks over the features)
//   gW2^T [64 x 64]  = h1^T dh2   gW3^T [64 x 32] = h2^T dy
// with M = 128 rows of which the rows past 288 / 64 are discarded. Their FP32
// accumulators stay in tensor memory over all tiles of the block. The bias
// gradients are FP32 column sums of dy, dh2, dh1 (warp shuffles, then per-warp
// sums in shared memory in a fixed order), so repeated runs agree bit for bit.
//
// TMEM (512 columns, 64-column blocks): gW1^T at 0 .. 191, gW2^T at 192,
// gW3^T at 256; layer 1 at 320, then h1 in FP32 (for 1 - h1^2); layer 2 at
// 384, then h2 in FP32, then dh2 W2; layer 3 at 448, then dy W3.
#include <cstdint>

#include "lbrr_launch.h"
#include "lbrr_mlp.h"
#include "lbrr_act.cuh"
#include "lbrr_tc.cuh"

namespace lbrr {

namespace {

using namespace tc;

constexpr int kRows = kMlpTrainRows;  // 128
constexpr int kThreads = 2 * kRows;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColG1 = 0, kColG2 = 192, kColG3 = 256, kColL1 = 320, kColL2 = 384,
                   kColL3 = 448;

// shared memory (bytes); every tile in the canonical K-major layout of its rows
constexpr uint32_t kSmW1 = 0;                                     // [64][288]
constexpr uint32_t kSmW2 = kSmW1 + kMlpHidden * kMlpIn * 2;      // [64][64]
constexpr uint32_t kSmW3 = kSmW2 + kMlpHidden * kMlpHidden * 2;  // [32][64]
constexpr uint32_t kSmW2t = kSmW3 + kMlpOut * kMlpHidden * 2;    // [64][64] = W2^T
constexpr uint32_t kSmW3t = kSmW2t + kMlpHidden * kMlpHidden * 2;  // [64][32] = W3^T
constexpr uint32_t kSmX = kSmW3t + kMlpHidden * kMlpOut * 2;     // [128][288]
constexpr uint32_t kSmH1 = kSmX + kRows * kMlpIn * 2;            // [128][64]
constexpr uint32_t kSmH2 = kSmH1 + kRows * kMlpHidden * 2;       // [128][64]
constexpr uint32_t kSmDy = kSmH2 + kRows * kMlpHidden * 2;       // [128][32]
constexpr uint32_t kSmDh2 = kSmDy + kRows * kMlpOut * 2;         // [128][64]
constexpr uint32_t kSmDh1 = kSmDh2 + kRows * kMlpHidden * 2;     // [128][64]
constexpr uint32_t kSmMisc = kSmDh1 + kRows * kMlpHidden * 2;
// misc: mbarrier, TMEM address, biases b1 b2 b3 (160), per-warp column sums of
// dy, dh2, dh1 (8 warps x 80 columns: a warp covers 32 rows and one half of
// the columns) and per-warp loss sums
constexpr int kGbCols = kMlpOut / 2 + kMlpHidden / 2 + kMlpHidden / 2;  // 80 per half
constexpr uint32_t kSmBias = kSmMisc + 64;
constexpr uint32_t kSmGbw = kSmBias + 4 * (2 * kMlpHidden + kMlpOut);
constexpr uint32_t kSmLossw = kSmGbw + 4 * 8 * kGbCols;
constexpr uint32_t kTrainSmem = kSmLossw + 4 * 8;
static_assert(kSmX % 1024 == 0 && kSmMisc % 16 == 0, "alignment");
static_assert(kTrainSmem <= 232448, "fits the shared memory of one block");
// the transposed reads with M = 128 run past the 288 (X) or 64 (h1, h2) real
// rows into the next tile's bytes (discarded rows): they stay inside the block
static_assert(kSmX + 15 * 36 * 128 + 47 * 128 + 36 * 128 + 128 <= kTrainSmem, "X^T reads");
static_assert(kSmH2 + 15 * 1024 + 15 * 128 + 1024 + 128 <= kTrainSmem, "h^T reads");

__host__ __device__ constexpr uint32_t idesc_t(int M, int N) {  // both operands MN-major
  return idesc_bf16(M, N) | (1u << 15) | (1u << 16);
}

// Operand descriptors of a [rows][C] tile (canonical, K-major rows): read
// K-major (K = C, the rows are M or N) or MN-major (K = rows, MN = C).
__device__ __forceinline__ uint64_t kmaj(uint32_t base, int C, int ks) {
  return sdesc(base + 256 * ks, 128, (C / 8) * 128);  // K step ks: 16 columns
}
__device__ __forceinline__ uint64_t mnmaj(uint32_t base, int C, int ks, int mn0 = 0) {
  // K step ks: rows 16 ks .. 16 ks + 15 (two 8-row groups); MN from column mn0
  return sdesc(base + 2 * ks * (C / 8) * 128 + (mn0 / 8) * 128, (C / 8) * 128, 128);
}

// 32 consecutive FP32 TMEM columns of this thread's lane into v
__device__ __forceinline__ void ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t a[16], b[16];
  tmem_ld16_async(taddr, a);
  tmem_ld16_async(taddr + 16, b);
  tmem_wait_ld();
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    v[k] = __uint_as_float(a[k]);
    v[16 + k] = __uint_as_float(b[k]);
  }
}
__device__ __forceinline__ void st32(uint32_t taddr, const float (&v)[32]) {
  uint32_t a[16], b[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    a[k] = __float_as_uint(v[k]);
    b[k] = __float_as_uint(v[16 + k]);
  }
  tmem_st16(taddr, a);
  tmem_st16(taddr + 16, b);
}
// values v[0 .. 8 NC) as BF16 into columns c0 .. of row r of a [rows][C] tile
template <int NC>
__device__ __forceinline__ void put_bf16(unsigned char *tile, int C, int r, int c0,
                                         const float *v) {
#pragma unroll
  for (int k = 0; k < 8 * NC; k += 8)
    *reinterpret_cast<uint4 *>(tile + cm_offset(r, c0 + k, C)) =
        make_uint4(pack_bf16(v[k], v[k + 1]), pack_bf16(v[k + 2], v[k + 3]),
                   pack_bf16(v[k + 4], v[k + 5]), pack_bf16(v[k + 6], v[k + 7]));
}
// column sums over the warp's 32 rows, added (lane 0) to dst[0 .. N)
template <int N>
__device__ __forceinline__ void warp_col_sums(const float *v, float *dst, int lane) {
#pragma unroll
  for (int k = 0; k < N; ++k) {
    float s = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) dst[k] += s;
  }
}

template <bool TRACE>
__global__ void __launch_bounds__(kThreads, 1)
    mlp_train_tc_kernel(MlpDevice p, const __nv_bfloat16 *__restrict__ X,
                        const float *__restrict__ T, long long M, float *__restrict__ gpart,
                        float *__restrict__ lpart, int *status, float *__restrict__ trace) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r = tid & (kRows - 1), half = tid >> 7;
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + kSmMisc);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kSmMisc + 8);
  float *sb = reinterpret_cast<float *>(smem + kSmBias);
  float *gbw = reinterpret_cast<float *>(smem + kSmGbw) + warp * kGbCols;
  float *lossw = reinterpret_cast<float *>(smem + kSmLossw);
  const uint32_t mbar_a = smem_u32(mbar);

  // ---- weights (and the transposed copies of W2, W3) in the canonical layout
  for (int c = tid; c < kMlpHidden * (kMlpIn / 8); c += kThreads) {
    const int n = c / (kMlpIn / 8), kb = c - n * (kMlpIn / 8);
    *reinterpret_cast<uint4 *>(smem + kSmW1 + cm_offset(n, 8 * kb, kMlpIn)) =
        *reinterpret_cast<const uint4 *>(p.w1 + n * kMlpIn + 8 * kb);
  }
  for (int c = tid; c < kMlpHidden * (kMlpHidden / 8); c += kThreads) {
    const int n = c / (kMlpHidden / 8), kb = c - n * (kMlpHidden / 8);
    *reinterpret_cast<uint4 *>(smem + kSmW2 + cm_offset(n, 8 * kb, kMlpHidden)) =
        *reinterpret_cast<const uint4 *>(p.w2 + n * kMlpHidden + 8 * kb);
    *reinterpret_cast<uint4 *>(smem + kSmW2t + cm_offset(n, 8 * kb, kMlpHidden)) =
        *reinterpret_cast<const uint4 *>(p.w2t + n * kMlpHidden + 8 * kb);
  }
  for (int c = tid; c < kMlpOut * (kMlpHidden / 8); c += kThreads) {
    const int n = c / (kMlpHidden / 8), kb = c - n * (kMlpHidden / 8);
    *reinterpret_cast<uint4 *>(smem + kSmW3 + cm_offset(n, 8 * kb, kMlpHidden)) =
        *reinterpret_cast<const uint4 *>(p.w3 + n * kMlpHidden + 8 * kb);
  }
  for (int c = tid; c < kMlpHidden * (kMlpOut / 8); c += kThreads) {
    const int n = c / (kMlpOut / 8), kb = c - n * (kMlpOut / 8);
    *reinterpret_cast<uint4 *>(smem + kSmW3t + cm_offset(n, 8 * kb, kMlpOut)) =
        *reinterpret_cast<const uint4 *>(p.w3t + n * kMlpOut + 8 * kb);
  }
  for (int c = tid; c < 2 * kMlpHidden + kMlpOut; c += kThreads)
    sb[c] = c < kMlpHidden ? p.b1[c] : (c < 2 * kMlpHidden ? p.b2[c - kMlpHidden]
                                                           : p.b3[c - 2 * kMlpHidden]);
  for (int c = tid; c < 8 * kGbCols; c += kThreads)
    reinterpret_cast<float *>(smem + kSmGbw)[c] = 0.f;
  if (tid < 8) lossw[tid] = 0.f;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar_a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t lane_addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
  const uint32_t sw1 = smem_u32(smem + kSmW1), sw2 = smem_u32(smem + kSmW2);
  const uint32_t sw3 = smem_u32(smem + kSmW3), sw2t = smem_u32(smem + kSmW2t);
  const uint32_t sw3t = smem_u32(smem + kSmW3t), sx = smem_u32(smem + kSmX);
  const uint32_t sh1 = smem_u32(smem + kSmH1), sh2 = smem_u32(smem + kSmH2);
  const uint32_t sdy = smem_u32(smem + kSmDy), sdh2 = smem_u32(smem + kSmDh2);
  const uint32_t sdh1 = smem_u32(smem + kSmDh1);
  const uint32_t lim = wait_limit(status);
  const float inv_n = 1.0f / ((float)M * (float)kMlpOutUsed);
  const long long ntiles = (M + kRows - 1) / kRows;
  uint32_t phase = 0;
  bool ok = true;
  // all threads wait for the MMAs committed so far (the same decision in every thread)
  auto sync_mma = [&]() {
    ok = !__syncthreads_or(!mbar_wait(mbar_a, phase, lim));
    phase ^= 1;
    fence_after();
    return ok;
  };
  auto handoff = [&]() {  // shared-memory and TMEM writes of every thread before the next MMAs
    tmem_wait_st();
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
  };

  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const bool first = tile == blockIdx.x;
    const long long row = tile * kRows + r;
    const bool valid = row < M;
    float *trow = TRACE && valid ? trace + row * kMlpTrace : nullptr;
    // ---- input rows: every 16-byte chunk of the thread's half row in flight
    // at once (cp.async), zeros past M
#pragma unroll
    for (int kb = half * (kMlpIn / 16); kb < (half + 1) * (kMlpIn / 16); ++kb) {
      unsigned char *dst = smem + kSmX + cm_offset(r, 8 * kb, kMlpIn);
      if (valid)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)),
                     "l"(X + row * kMlpIn + 8 * kb)
                     : "memory");
      else
        *reinterpret_cast<uint4 *>(dst) = make_uint4(0u, 0u, 0u, 0u);
    }
    cp_async_wait_all();
    handoff();
    // ---- layer 1
    if (tid == 0) {
#pragma unroll 1
      for (int ks = 0; ks < kMlpIn / 16; ++ks)
        umma(tmem + kColL1, kmaj(sx, kMlpIn, ks), kmaj(sw1, kMlpIn, ks),
             idesc_bf16(128, kMlpHidden), ks > 0);
      umma_commit(mbar_a);
    }
    if (!sync_mma()) break;
    float v[32];
    ld32(lane_addr + kColL1 + 32 * half, v);
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = tanh_approx(v[k] + sb[32 * half + k]);
    st32(lane_addr + kColL1 + 32 * half, v);  // h1 in FP32, for 1 - h1^2
    put_bf16<4>(smem + kSmH1, kMlpHidden, r, 32 * half, v);
    if (TRACE && trow)
#pragma unroll
      for (int k = 0; k < 32; ++k) trow[kTraceH1 + 32 * half + k] = v[k];
    handoff();
    // ---- layer 2
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < kMlpHidden / 16; ++ks)
        umma(tmem + kColL2, kmaj(sh1, kMlpHidden, ks), kmaj(sw2, kMlpHidden, ks),
             idesc_bf16(128, kMlpHidden), ks > 0);
      umma_commit(mbar_a);
    }
    if (!sync_mma()) break;
    ld32(lane_addr + kColL2 + 32 * half, v);
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = tanh_approx(v[k] + sb[kMlpHidden + 32 * half + k]);
    st32(lane_addr + kColL2 + 32 * half, v);  // h2 in FP32
    put_bf16<4>(smem + kSmH2, kMlpHidden, r, 32 * half, v);
    if (TRACE && trow)
#pragma unroll
      for (int k = 0; k < 32; ++k) trow[kTraceH2 + 32 * half + k] = v[k];
    handoff();
    // ---- layer 3, loss and dy (this thread: outputs 16 half .. 16 half + 15)
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < kMlpHidden / 16; ++ks)
        umma(tmem + kColL3, kmaj(sh2, kMlpHidden, ks), kmaj(sw3, kMlpHidden, ks),
             idesc_bf16(128, kMlpOut), ks > 0);
      umma_commit(mbar_a);
    }
    if (!sync_mma()) break;
    {
      uint32_t a[16];
      tmem_ld16_async(lane_addr + kColL3 + 16 * half, a);
      tmem_wait_ld();
      float dy[16], lsum = 0.f;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int o = 16 * half + k;
        const float y = __uint_as_float(a[k]) + sb[2 * kMlpHidden + o];
        const float d = valid && o < kMlpOutUsed ? y - T[row * kMlpOut + o] : 0.f;
        lsum = fmaf(d, d, lsum);
        dy[k] = 2.0f * d * inv_n;
        if (TRACE && trow) {
          trow[kTraceY + o] = y;
          trow[kTraceDy + o] = dy[k];
        }
      }
      put_bf16<2>(smem + kSmDy, kMlpOut, r, 16 * half, dy);
      warp_col_sums<16>(dy, gbw, lane);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
      if (lane == 0) lossw[warp] += lsum;
    }
    handoff();
    // ---- dh2 = (dy W3) (1 - h2^2): K = 32 over the outputs, into layer 3's columns
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < kMlpOut / 16; ++ks)
        umma(tmem + kColL3, kmaj(sdy, kMlpOut, ks), kmaj(sw3t, kMlpOut, ks),
             idesc_bf16(128, kMlpHidden), ks > 0);
      umma_commit(mbar_a);
    }
    if (!sync_mma()) break;
    {
      float hv[32];
      ld32(lane_addr + kColL3 + 32 * half, v);
      ld32(lane_addr + kColL2 + 32 * half, hv);
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] *= 1.0f - hv[k] * hv[k];
      put_bf16<4>(smem + kSmDh2, kMlpHidden, r, 32 * half, v);
      if (TRACE && trow)
#pragma unroll
        for (int k = 0; k < 32; ++k) trow[kTraceDh2 + 32 * half + k] = v[k];
      warp_col_sums<32>(v, gbw + kMlpOut / 2, lane);
    }
    handoff();
    // ---- dh1 = (dh2 W2) (1 - h1^2), into layer 2's columns (h2 is no longer needed)
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < kMlpHidden / 16; ++ks)
        umma(tmem + kColL2, kmaj(sdh2, kMlpHidden, ks), kmaj(sw2t, kMlpHidden, ks),
             idesc_bf16(128, kMlpHidden), ks > 0);
      umma_commit(mbar_a);
    }
    if (!sync_mma()) break;
    {
      float hv[32];
      ld32(lane_addr + kColL2 + 32 * half, v);
      ld32(lane_addr + kColL1 + 32 * half, hv);
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] *= 1.0f - hv[k] * hv[k];
      put_bf16<4>(smem + kSmDh1, kMlpHidden, r, 32 * half, v);
      if (TRACE && trow)
#pragma unroll
        for (int k = 0; k < 32; ++k) trow[kTraceDh1 + 32 * half + k] = v[k];
      warp_col_sums<32>(v, gbw + kMlpOut / 2 + kMlpHidden / 2, lane);
    }
    handoff();
    // ---- weight gradients, K = the tile's 128 rows, accumulated over the tiles
    if (tid == 0) {
#pragma unroll 1
      for (int ks = 0; ks < kRows / 16; ++ks) {
        const uint32_t acc = !first || ks > 0;
#pragma unroll
        for (int q = 0; q < 3; ++q)
          umma(tmem + kColG1 + 64 * q, mnmaj(sx, kMlpIn, ks, 128 * q),
               mnmaj(sdh1, kMlpHidden, ks), idesc_t(128, kMlpHidden), acc);
        umma(tmem + kColG2, mnmaj(sh1, kMlpHidden, ks), mnmaj(sdh2, kMlpHidden, ks),
             idesc_t(128, kMlpHidden), acc);
        umma(tmem + kColG3, mnmaj(sh2, kMlpHidden, ks), mnmaj(sdy, kMlpOut, ks),
             idesc_t(128, kMlpOut), acc);
      }
      umma_commit(mbar_a);
    }
    if (!sync_mma()) break;  // the next tile overwrites the operand tiles
  }

  if (ok) {
    // ---- block partials in the packed parameter order: thread (r, half)
    // holds lane r of each accumulator and half of its columns
    float *o = gpart + (long long)blockIdx.x * kMlpParams;
    float v[32];
#pragma unroll 1
    for (int q = 0; q < 3; ++q) {  // gW1[j][f], f = 128 q + r
      ld32(lane_addr + kColG1 + 64 * q + 32 * half, v);
      const int f = 128 * q + r;
      if (f < kMlpIn)
#pragma unroll
        for (int k = 0; k < 32; ++k) o[kOffW1 + (32 * half + k) * kMlpIn + f] = v[k];
    }
    ld32(lane_addr + kColG2 + 32 * half, v);  // gW2[j][i], i = r
    if (r < kMlpHidden)
#pragma unroll
      for (int k = 0; k < 32; ++k) o[kOffW2 + (32 * half + k) * kMlpHidden + r] = v[k];
    {
      uint32_t a[16];  // gW3[o][j], j = r
      tmem_ld16_async(lane_addr + kColG3 + 16 * half, a);
      tmem_wait_ld();
      if (r < kMlpHidden)
#pragma unroll
        for (int k = 0; k < 16; ++k)
          o[kOffW3 + (16 * half + k) * kMlpHidden + r] = __uint_as_float(a[k]);
    }
    __syncthreads();
    // bias gradients: the four row warps of each half, in order
    const float *g = reinterpret_cast<const float *>(smem + kSmGbw);
    for (int c = tid; c < 2 * kGbCols; c += kThreads) {
      const int h = c / kGbCols, k = c - h * kGbCols;
      const float s = ((g[(4 * h + 0) * kGbCols + k] + g[(4 * h + 1) * kGbCols + k]) +
                       g[(4 * h + 2) * kGbCols + k]) +
                      g[(4 * h + 3) * kGbCols + k];
      if (k < kMlpOut / 2)
        o[kOffB3 + 16 * h + k] = s;
      else if (k < kMlpOut / 2 + kMlpHidden / 2)
        o[kOffB2 + 32 * h + k - kMlpOut / 2] = s;
      else
        o[kOffB1 + 32 * h + k - kMlpOut / 2 - kMlpHidden / 2] = s;
    }
    if (tid == 0)
      lpart[blockIdx.x] = (((lossw[0] + lossw[1]) + (lossw[2] + lossw[3])) +
                           ((lossw[4] + lossw[5]) + (lossw[6] + lossw[7])));
  } else {
    if (tid == 0) atomicExch(status, 1);
    mbar_wait(mbar_a, phase);  // MMAs still in flight finish before the memory goes away
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
}

}  // namespace

cudaError_t launch_mlp_train(const MlpDevice &p, const void *X, const float *T, long long M,
                             float *gpart, float *lpart, int *status, int nblocks,
                             cudaStream_t st, float *trace) {
  if (!T || M < 1) return cudaErrorInvalidValue;
  auto kern = trace ? mlp_train_tc_kernel<true> : mlp_train_tc_kernel<false>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem);
  if (e != cudaSuccess) return e;
  const long long tiles = (M + kRows - 1) / kRows;
  const int nb = (int)(tiles < nblocks ? tiles : nblocks);
  kern<<<nb, kThreads, kTrainSmem, st>>>(p, static_cast<const __nv_bfloat16 *>(X), T, M, gpart,
                                         lpart, status, trace);
  return cudaGetLastError();
}

}  // namespace lbrr
