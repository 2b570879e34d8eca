// Forward pass of the closure network on the 5th-generation tensor cores
// (tcgen05, sm_100-family): y = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3 for
// tiles of 128 rows, BF16 operands in shared memory, FP32 accumulators in
// tensor memory (TMEM).
//
// One block per SM (persistent). The BF16 weights are staged once into shared
// memory in the canonical K-major layout without swizzle: 8 x 8 "core
// matrices" of 128 contiguous bytes (8 rows of 16 bytes), adjacent core
// matrices along K 128 bytes apart (leading byte offset) and adjacent 8-row
// groups K/8 * 128 bytes apart (stride byte offset). Per tile the 128 threads
// write the 128 input rows (thread r owns row r = TMEM lane r) in the same
// layout; one thread issues the K/16 MMAs of a layer (M = 128, N = 64, 64, 32)
// and commits them to an mbarrier; the threads then read their row of the
// accumulator (tcgen05.ld 32x32b), add the bias, apply tanh, round to BF16 and
// write the next layer's input rows. TMEM columns: layer 1 at 0, layer 2 at 64,
// layer 3 at 128 (256 allocated).
//
// Every mbarrier wait is bounded: on expiry the block records a timeout in
// *status, waits (bounded) for its MMAs to drain, frees its TMEM and returns.
#include <cstdint>

#include "lbrr_launch.h"
#include "lbrr_mlp.h"
#include "lbrr_act.cuh"
#include "lbrr_tc.cuh"

namespace lbrr {

namespace {

using namespace tc;

constexpr int kTcRows = 128;
constexpr int kTcThreads = 256;  // two threads per row; warps w and w + 4 share TMEM lanes
constexpr uint32_t kTmemCols = 256;

// shared-memory plan (bytes, all 1024-aligned)
constexpr uint32_t kW1Bytes = kMlpHidden * kMlpIn * 2;        // 36864
constexpr uint32_t kW2Bytes = kMlpHidden * kMlpHidden * 2;    // 8192
constexpr uint32_t kW3Bytes = kMlpOut * kMlpHidden * 2;       // 4096
constexpr uint32_t kA1Bytes = kTcRows * kMlpIn * 2;           // 73728
constexpr uint32_t kA2Bytes = kTcRows * kMlpHidden * 2;       // 16384
constexpr uint32_t kOffSW1 = 0;
constexpr uint32_t kOffSW2 = kOffSW1 + kW1Bytes;
constexpr uint32_t kOffSW3 = kOffSW2 + kW2Bytes;
constexpr uint32_t kOffSA1 = kOffSW3 + kW3Bytes;
constexpr uint32_t kOffSA2 = kOffSA1 + kA1Bytes;
constexpr uint32_t kOffSA3 = kOffSA2 + kA2Bytes;
constexpr uint32_t kOffMisc = kOffSA3 + kA2Bytes;  // mbarrier, TMEM address, biases
// staged moment field of a row-segment tile: 9 neighbour rows x 10 moments,
// x0 - 1 .. x0 + 128 at positions 3 .. 132 (interior 16-byte aligned at 4)
constexpr int kMsLen = 136;
constexpr uint32_t kOffMs = kOffMisc + 1024;
constexpr uint32_t kMsBytes = 9 * kMlpMoments * kMsLen * 4;  // 48960
constexpr uint32_t kTcSmem = kOffMs + kMsBytes;

__device__ __forceinline__ uint32_t pack2(float lo, float hi) { return pack_bf16(lo, hi); }

// Layer epilogue: tanh(acc + bias) of 32 of the 64 columns (half 0 or 1) into
// row r of a K = 64 operand; with TRACE also the FP32 values into hrow[64].
template <bool TRACE = false>
__device__ __forceinline__ void hidden_epilogue(uint32_t taddr, const float *bias,
                                                unsigned char *dst, int r, int half,
                                                float *hrow = nullptr) {
#pragma unroll
  for (int c0 = 32 * half; c0 < 32 * half + 32; c0 += 16) {
    float v[16];
    tmem_ld16(taddr + c0, v);
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = tanh_approx(v[k] + bias[c0 + k]);
    if (TRACE && hrow)
#pragma unroll
      for (int k = 0; k < 16; k += 4)
        *reinterpret_cast<float4 *>(hrow + c0 + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
#pragma unroll
    for (int k = 0; k < 16; k += 8) {
      uint4 q;
      q.x = pack2(v[k], v[k + 1]);
      q.y = pack2(v[k + 2], v[k + 3]);
      q.z = pack2(v[k + 4], v[k + 5]);
      q.w = pack2(v[k + 6], v[k + 7]);
      *reinterpret_cast<uint4 *>(dst + cm_offset(r, c0 + k, kMlpHidden)) = q;
    }
  }
}

// Standardised feature f = 10 nb + k of row r from the staged moment rows
// ms[row9 * 10 + k] (row9 = (dy+1) + 3 (dz+1)) at x offset 4 + r + dx.
template <int F>
__device__ __forceinline__ float staged_feature(const MlpDevice &p, const float *ms, int r) {
  constexpr int nb = F / kMlpMoments, k = F % kMlpMoments;
  constexpr int dx = nb % 3 - 1, row9 = nb / 3;
  return (ms[(row9 * kMlpMoments + k) * kMsLen + 4 + r + dx] - p.in_mean[k]) * p.in_inv_std[k];
}

template <int F>
__device__ __forceinline__ uint32_t staged_pair(const MlpDevice &p, const float *ms, int r) {
  if constexpr (F >= kMlpInUsed)
    return 0u;
  else
    return pack2(staged_feature<F>(p, ms, r), staged_feature<F + 1>(p, ms, r));
}

// Chunks KB0 .. KB0 + 17 (8 features each) of row r, as 16-byte stores.
template <int KB0, int KB = KB0>
__device__ __forceinline__ void staged_chunks(const MlpDevice &p, const float *ms,
                                              unsigned char *a1, int r) {
  if constexpr (KB < KB0 + kMlpIn / 16) {
    uint4 q;
    q.x = staged_pair<8 * KB>(p, ms, r);
    q.y = staged_pair<8 * KB + 2>(p, ms, r);
    q.z = staged_pair<8 * KB + 4>(p, ms, r);
    q.w = staged_pair<8 * KB + 6>(p, ms, r);
    *reinterpret_cast<uint4 *>(a1 + cm_offset(r, 8 * KB, kMlpIn)) = q;
    staged_chunks<KB0, KB + 1>(p, ms, a1, r);
  }
}

// Features of row r into the A1 tile: half 0 writes chunks 0..17, half 1
// chunks 18..35 (the last ones hold the zero padding).
__device__ __forceinline__ void features_staged(const MlpDevice &p, const float *ms,
                                                unsigned char *a1, int r, int half) {
  if (half == 0)
    staged_chunks<0>(p, ms, a1, r);
  else
    staged_chunks<kMlpIn / 16>(p, ms, a1, r);
}

// Same from the moment field in global memory (any grid shape).
__device__ __forceinline__ void features_gather(const MlpDevice &p, const float *mom,
                                                const Grid &g, long long cell,
                                                unsigned char *a1, int r, int half) {
  int x, y, z;
  cell_coords(cell, g, x, y, z);
  const long long n = g.n;
#pragma unroll 1
  for (int nb = half ? 14 : 0; nb < (half ? 27 : 14); ++nb) {
    const int dx = nb % 3 - 1, dy = (nb / 3) % 3 - 1, dz = nb / 9 - 1;
    const long long c = ((long long)wrap_add(z, dz, g.nz) * g.ny + wrap_add(y, dy, g.ny)) * g.nx +
                        wrap_add(x, dx, g.nx);
#pragma unroll
    for (int k = 0; k < kMlpMoments; k += 2) {
      const float v0 = (__ldg(mom + k * n + c) - p.in_mean[k]) * p.in_inv_std[k];
      const float v1 = (__ldg(mom + (k + 1) * n + c) - p.in_mean[k + 1]) * p.in_inv_std[k + 1];
      *reinterpret_cast<uint32_t *>(a1 + cm_offset(r, kMlpMoments * nb + k, kMlpIn)) =
          pack2(v0, v1);
    }
  }
  if (half)
    for (int f = kMlpInUsed; f < kMlpIn; f += 2)
      *reinterpret_cast<uint32_t *>(a1 + cm_offset(r, f, kMlpIn)) = 0u;
}

// FROM_MOM: rows are the cells of a grid and their features are built from
// the moment field mom [10][N]; outputs y[k][cell] for the 17 used outputs.
// When nx is a multiple of 128 a tile is one row segment and the 9 x 10
// moment rows around it are first staged in shared memory with 16-byte loads.
// Otherwise rows are X [M][288] (BF16) and outputs Y [M][32].
// TRACE (rows X only): also H[row][0..63] and H[row][64..127], the FP32
// activations of layers 1 and 2 before their BF16 rounding.
template <bool FROM_MOM, bool TRACE = false>
__global__ void __launch_bounds__(kTcThreads, 1)
    mlp_tc_kernel(MlpDevice p, const __nv_bfloat16 *__restrict__ X,
                  const float *__restrict__ mom, const Grid g, long long M,
                  float *__restrict__ Y, int *status, float *__restrict__ H) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int r = tid & (kTcRows - 1), half = tid >> 7;  // row, and which half of its work
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + kOffMisc);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kOffMisc + 8);
  float *sb = reinterpret_cast<float *>(smem + kOffMisc + 64);  // b1, b2, b3 (160)
  float *ms = reinterpret_cast<float *>(smem + kOffMs);
  const uint32_t mbar_a = smem_u32(mbar);

  // ---- weights into the canonical layout; biases
  for (int c = tid; c < kMlpHidden * (kMlpIn / 8); c += kTcThreads) {
    const int n = c / (kMlpIn / 8), kb = c - n * (kMlpIn / 8);
    *reinterpret_cast<uint4 *>(smem + kOffSW1 + cm_offset(n, 8 * kb, kMlpIn)) =
        *reinterpret_cast<const uint4 *>(p.w1 + n * kMlpIn + 8 * kb);
  }
  for (int c = tid; c < kMlpHidden * (kMlpHidden / 8); c += kTcThreads) {
    const int n = c / (kMlpHidden / 8), kb = c - n * (kMlpHidden / 8);
    *reinterpret_cast<uint4 *>(smem + kOffSW2 + cm_offset(n, 8 * kb, kMlpHidden)) =
        *reinterpret_cast<const uint4 *>(p.w2 + n * kMlpHidden + 8 * kb);
  }
  for (int c = tid; c < kMlpOut * (kMlpHidden / 8); c += kTcThreads) {
    const int n = c / (kMlpHidden / 8), kb = c - n * (kMlpHidden / 8);
    *reinterpret_cast<uint4 *>(smem + kOffSW3 + cm_offset(n, 8 * kb, kMlpHidden)) =
        *reinterpret_cast<const uint4 *>(p.w3 + n * kMlpHidden + 8 * kb);
  }
  for (int c = tid; c < 2 * kMlpHidden + kMlpOut; c += kTcThreads)
    sb[c] = c < kMlpHidden ? p.b1[c] : (c < 2 * kMlpHidden ? p.b2[c - kMlpHidden]
                                                           : p.b3[c - 2 * kMlpHidden]);
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
  // TMEM lanes of this warp: 32 (warp % 4) ..
  const uint32_t lane_addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16);

  const uint32_t sw1 = smem_u32(smem + kOffSW1), sw2 = smem_u32(smem + kOffSW2);
  const uint32_t sw3 = smem_u32(smem + kOffSW3), sa1 = smem_u32(smem + kOffSA1);
  const uint32_t sa2 = smem_u32(smem + kOffSA2), sa3 = smem_u32(smem + kOffSA3);
  uint32_t phase = 0;
  bool ok = true;
  const long long ntiles = (M + kTcRows - 1) / kTcRows;
  const long long n = g.n;
  const bool staged = FROM_MOM && (g.nx % kTcRows == 0);

  // asynchronous copy of the 9 x 10 moment rows around a row-segment tile
  // (x0 - 1 .. x0 + 128, periodic) into ms
  auto stage = [&](long long t) {
    const long long first = t * kTcRows;
    const int x0 = (int)(first % g.nx);
    const long long yz = first / g.nx;
    const int y = (int)(yz % g.ny), z = (int)(yz / g.ny);
    for (int q = tid; q < 9 * kMlpMoments * (kTcRows / 4); q += kTcThreads) {
      const int sgm = q / (kTcRows / 4), j = q - sgm * (kTcRows / 4);
      const int row9 = sgm / kMlpMoments, k = sgm - row9 * kMlpMoments;
      const int yy = wrap_add(y, row9 % 3 - 1, g.ny), zz = wrap_add(z, row9 / 3 - 1, g.nz);
      const float *src = mom + k * n + ((long long)zz * g.ny + yy) * g.nx + x0 + 4 * j;
      const unsigned d = smem_u32(ms + sgm * kMsLen + 4 + 4 * j);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
    }
    for (int q = tid; q < 9 * kMlpMoments * 2; q += kTcThreads) {
      const int sgm = q >> 1, side = q & 1;
      const int row9 = sgm / kMlpMoments, k = sgm - row9 * kMlpMoments;
      const int yy = wrap_add(y, row9 % 3 - 1, g.ny), zz = wrap_add(z, row9 / 3 - 1, g.nz);
      const int xx = side ? (x0 + kTcRows == g.nx ? 0 : x0 + kTcRows)
                          : (x0 == 0 ? g.nx - 1 : x0 - 1);
      const float *src = mom + k * n + ((long long)zz * g.ny + yy) * g.nx + xx;
      const unsigned d = smem_u32(ms + sgm * kMsLen + (side ? 4 + kTcRows : 3));
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
    }
  };
  if (staged && (long long)blockIdx.x < ntiles) stage(blockIdx.x);

  for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const long long row = tile * kTcRows + r;
    const bool valid = row < M;
    unsigned char *a1 = smem + kOffSA1;
    // ---- input rows
    if (FROM_MOM && staged) {
      // the moment rows of this tile were requested (cp.async) before the
      // previous tile's products; wait for them, build the features, then
      // request the next tile's rows so that they arrive during this tile's
      // products and epilogues
      asm volatile("cp.async.wait_all;\n" ::: "memory");
      __syncthreads();
      features_staged(p, ms, a1, r, half);
      __syncthreads();
      if (tile + gridDim.x < ntiles) stage(tile + gridDim.x);
    } else if (FROM_MOM) {
      if (valid) {
        features_gather(p, mom, g, row, a1, r, half);
      } else {
        for (int kb = half * (kMlpIn / 16); kb < (half + 1) * (kMlpIn / 16); ++kb)
          *reinterpret_cast<uint4 *>(a1 + cm_offset(r, 8 * kb, kMlpIn)) =
              make_uint4(0u, 0u, 0u, 0u);
      }
    } else {
#pragma unroll 3
      for (int kb = half * (kMlpIn / 16); kb < (half + 1) * (kMlpIn / 16); ++kb) {
        const uint4 q = valid ? *reinterpret_cast<const uint4 *>(X + row * kMlpIn + 8 * kb)
                              : make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4 *>(a1 + cm_offset(r, 8 * kb, kMlpIn)) = q;
      }
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    // ---- layer 1: D[128 x 64] (TMEM cols 0..63) = A1[128 x 288] W1^T
    if (tid == 0) {
#pragma unroll 1
      for (int ks = 0; ks < kMlpIn / 16; ++ks)
        umma(tmem, sdesc(sa1 + 256 * ks, 128, (kMlpIn / 8) * 128),
             sdesc(sw1 + 256 * ks, 128, (kMlpIn / 8) * 128), idesc_bf16(128, 64), ks > 0);
      umma_commit(mbar_a);
    }
    ok = !__syncthreads_or(!mbar_wait(mbar_a, phase));  // same decision in every thread
    phase ^= 1;
    fence_after();
    if (!ok) break;
    hidden_epilogue<TRACE>(lane_addr + 0, sb, smem + kOffSA2, r, half,
                           TRACE && valid ? H + row * (2 * kMlpHidden) : nullptr);
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    // ---- layer 2 (TMEM cols 64..127)
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < kMlpHidden / 16; ++ks)
        umma(tmem + 64, sdesc(sa2 + 256 * ks, 128, (kMlpHidden / 8) * 128),
             sdesc(sw2 + 256 * ks, 128, (kMlpHidden / 8) * 128), idesc_bf16(128, 64), ks > 0);
      umma_commit(mbar_a);
    }
    ok = !__syncthreads_or(!mbar_wait(mbar_a, phase));
    phase ^= 1;
    fence_after();
    if (!ok) break;
    hidden_epilogue<TRACE>(lane_addr + 64, sb + kMlpHidden, smem + kOffSA3, r, half,
                           TRACE && valid ? H + row * (2 * kMlpHidden) + kMlpHidden : nullptr);
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    // ---- layer 3 (TMEM cols 128..159): each half reads 16 of the 32 columns
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < kMlpHidden / 16; ++ks)
        umma(tmem + 128, sdesc(sa3 + 256 * ks, 128, (kMlpHidden / 8) * 128),
             sdesc(sw3 + 256 * ks, 128, (kMlpHidden / 8) * 128), idesc_bf16(128, 32), ks > 0);
      umma_commit(mbar_a);
    }
    ok = !__syncthreads_or(!mbar_wait(mbar_a, phase));
    phase ^= 1;
    fence_after();
    if (!ok) break;
    float y[16];
    tmem_ld16(lane_addr + 128 + 16 * half, y);
    if (valid) {
      const float *b3 = sb + 2 * kMlpHidden + 16 * half;
      if (FROM_MOM) {
#pragma unroll
        for (int k = 0; k < 16; ++k)
          if (16 * half + k < kMlpOutUsed) Y[(16 * half + k) * M + row] = y[k] + b3[k];
      } else {
#pragma unroll
        for (int k = 0; k < 16; k += 4)
          *reinterpret_cast<float4 *>(Y + row * kMlpOut + 16 * half + k) =
              make_float4(y[k] + b3[k], y[k + 1] + b3[k + 1], y[k + 2] + b3[k + 2],
                          y[k + 3] + b3[k + 3]);
      }
    }
    fence_before();
    __syncthreads();  // the next tile overwrites A1, the staged moments and the accumulators
    fence_after();
  }

  asm volatile("cp.async.wait_all;\n" ::: "memory");  // no copy outlives the block
  if (!ok) {
    if (tid == 0) atomicExch(status, 1);
    // let any MMA still in flight finish before the memory goes away
    mbar_wait(mbar_a, phase);
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

cudaError_t launch_mlp_tc(const MlpDevice &p, const void *X, const float *mom, const Grid *g,
                          long long M, float *Y, int *status, int nblocks, cudaStream_t st,
                          float *H) {
  const bool from_mom = mom != nullptr;
  if (from_mom && H) return cudaErrorInvalidValue;
  auto kern = from_mom ? mlp_tc_kernel<true> : (H ? mlp_tc_kernel<false, true>
                                                  : mlp_tc_kernel<false>);
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
  if (e != cudaSuccess) return e;
  const long long tiles = (M + kTcRows - 1) / kTcRows;
  const int nb = (int)(tiles < nblocks ? tiles : nblocks);
  const Grid gg = g ? *g : Grid{1, 1, 1, M};
  kern<<<nb, kTcThreads, kTcSmem, st>>>(p, static_cast<const __nv_bfloat16 *>(X), mom, gg, M, Y,
                                        status, H);
  return cudaGetLastError();
}

}  // namespace lbrr
