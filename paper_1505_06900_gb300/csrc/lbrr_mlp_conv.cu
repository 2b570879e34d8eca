// Closure-network forward pass fused with the closure update, for grids whose
// rows are whole 128-cell tiles, fed by the tensor memory accelerator (TMA)
// and pipelined across tiles.
//
// Layer 1 of the network is a 3x3x3 convolution of the standardised moment
// field: its 270 inputs for a cell are the 10 moments of the 27 cells around
// it. A feature-source tensor holds those moments once per cell, standardised
// and rounded to BF16, channels-last with 16 channels (10 used) and a one-cell
// periodic halo: xs[z + 1][y + 1][x + 1][16]. For a tile of 128 cells
// x0 .. x0 + 127 of row (y, z) the kernel copies, per neighbour row
// (y + dy, z + dz), the 130 positions x0 - 1 .. x0 + 128 with two TMA tile
// loads (channels 0-7 and 8-15), which lands them as [130 rows][16 bytes]:
// the canonical K-major layout without swizzle (8-row groups 128 bytes
// apart, the two channel halves one row block apart). The 27 MMAs of layer
// 1 (M 128, N 64, K 16, one per neighbour (dx, dy, dz)) read that block
// starting dx + 1 rows in; the weight operand of each neighbour is W1's 10
// columns of that neighbour, zero-padded to 16.
//
// One persistent block per SM, eighteen warps:
//   warp 0      TMA producer: 18 tile loads per tile into one of 2 stages
//   warp 1      layer-1 MMA issuer (and TMEM owner)
//   warps 2-17  four epilogue groups of four warps taking every fourth tile;
//               each reads its layer-1 accumulator (thread = TMEM lane = tile
//               row), applies bias and tanh, writes the BF16 hidden row,
//               issues layers 2 and 3 itself and, with the 17 standardised
//               outputs of its row, performs the closure update of that
//               row's cell in the population store (closure_update_cell):
//               the step of the learned closure is fused into the network.
// Group g owns TMEM columns 128 g .. 128 g + 127: the first 64 take its
// layer-1 accumulator (released as soon as the group has read it, so the
// next tile's layer 1 can start), the other 64 its layer 2 and then layer 3.
// Every barrier is waited on by one role in the order of its phases.
// Stages, accumulators and epilogue groups are handed over with mbarriers;
// every wait is bounded (status[1] can shorten the main-loop limit to test
// the timeout path). On a timeout the block raises a shared abort flag,
// every role leaves its loop, copies and MMAs still in flight are waited for
// (bounded), the tensor memory is freed and *status is set to 1.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>

#include "lbrr_launch.h"
#include "lbrr_mlp.h"
#include "lbrr_mma.cuh"
#include "lbrr_tc.cuh"

namespace lbrr {

namespace {

using namespace tc;

constexpr int kCRows = 128;                         // cells per tile
constexpr int kCSpan = kCRows + 2;                  // staged positions x0 - 1 .. x0 + 128
constexpr uint32_t kHalfBytes = kCSpan * 16;        // one channel half of a neighbour row
constexpr uint32_t kHalfPitch = 2176;               // the same, 128-byte aligned
constexpr uint32_t kStageBytes = 18 * kHalfPitch;   // 9 neighbour rows x 2 halves
constexpr uint32_t kTxBytes = 18 * kHalfBytes;      // bytes a stage receives
constexpr int kStages = 2;
constexpr int kTaps = 27;
constexpr uint32_t kTapBytes = 2 * kMlpHidden * 16;  // W1 block of one neighbour
constexpr uint32_t kA2Bytes = kCRows * kMlpHidden * 2;
constexpr int kGroups = 4;                          // epilogue groups
constexpr int kConvThreads = 32 * (2 + 4 * kGroups);
constexpr uint32_t kTmemCols = 512;

constexpr uint32_t kOffW1 = 0;
constexpr uint32_t kOffW2 = kOffW1 + kTaps * kTapBytes;
constexpr uint32_t kOffW3 = kOffW2 + kMlpHidden * kMlpHidden * 2;
constexpr uint32_t kOffA1 = kOffW3 + kMlpOut * kMlpHidden * 2;
constexpr uint32_t kOffA2 = kOffA1 + kStages * kStageBytes;
constexpr uint32_t kOffMisc = kOffA2 + kGroups * kA2Bytes;
constexpr uint32_t kConvSmem = kOffMisc + 1024;
static_assert(kOffA1 % 128 == 0 && kStageBytes % 128 == 0 && kHalfPitch % 128 == 0,
              "TMA destinations are 128-byte aligned");
static_assert(kConvSmem <= 232448, "fits the shared memory of one block");

// mbarriers in the misc area
enum : int {
  kBarFull = 0,                       // [stages] stage loaded (TMA transaction bytes)
  kBarEmpty = kBarFull + kStages,     // [stages] stage consumed by the layer-1 MMAs
  kBarAcc1F = kBarEmpty + kStages,    // [groups] layer-1 accumulator ready (tcgen05.commit)
  kBarAcc1E = kBarAcc1F + kGroups,    // [groups] layer-1 accumulator read by its group
  kBarL2 = kBarAcc1E + kGroups,       // [groups] layer 2 done
  kBarL3 = kBarL2 + kGroups,          // [groups] layer 3 done
  kBarDrain = kBarL3 + kGroups,       // [1 + groups] drain of each MMA issuer after an abort
  kNumBars = kBarDrain + 1 + kGroups
};
static_assert(kNumBars * 8 + 16 <= 256, "barriers, TMEM slot and counters before the biases");

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes)
               : "memory");
}
// 4-D tiled TMA load (coordinates innermost first), completing on mbar
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, int c3, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mbar)
      : "memory");
}
// barrier of one epilogue group (4 warps, named barrier 1 + g)
__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, 128;\n" ::"r"(1 + g) : "memory");
}
// the same, returning whether any thread of the group passed pred = true
__device__ __forceinline__ bool group_any(int g, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, %2, 128, p;\n"
      "selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(1 + g)
      : "memory");
  return r != 0;
}

// tanh(acc + bias) of 32 accumulator columns c0 .. c0 + 31 (in v) into row r
// of a K = 64 operand (canonical layout), BF16; with TRACE also the FP32
// values into trace_row[c0 ..].
template <bool TRACE = false>
__device__ __forceinline__ void hidden_half(const uint32_t (&v)[32], const float *bias, int c0,
                                            unsigned char *dst, int r,
                                            float *trace_row = nullptr) {
#pragma unroll
  for (int k = 0; k < 32; k += 8) {
    float h[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) h[e] = tanh_approx(__uint_as_float(v[k + e]) + bias[c0 + k + e]);
    if (TRACE)
#pragma unroll
      for (int e = 0; e < 8; ++e) trace_row[c0 + k + e] = h[e];
    uint4 q;
    q.x = pack_bf16(h[0], h[1]);
    q.y = pack_bf16(h[2], h[3]);
    q.z = pack_bf16(h[4], h[5]);
    q.w = pack_bf16(h[6], h[7]);
    *reinterpret_cast<uint4 *>(dst + cm_offset(r, c0 + k, kMlpHidden)) = q;
  }
}

__device__ __forceinline__ void load_acc32(uint32_t taddr, uint32_t (&v)[32]) {
  uint32_t (&a)[16] = *reinterpret_cast<uint32_t(*)[16]>(&v[0]);
  uint32_t (&b)[16] = *reinterpret_cast<uint32_t(*)[16]>(&v[16]);
  tmem_ld16_async(taddr, a);
  tmem_ld16_async(taddr + 16, b);
  tmem_wait_ld();
}

// TRACE: also trace[cell][0..63], [64..127] (the FP32 activations of layers
// 1 and 2 before their BF16 rounding) and [128..144] (the 17 standardised
// predictions) of every cell.
template <int PARITY, typename IDX, bool TRACE = false>
__global__ void __launch_bounds__(kConvThreads, 1)
    mlp_conv_kernel(MlpDevice p, const __grid_constant__ CUtensorMap xs_map, const Grid g,
                    float *__restrict__ f, const float om1, unsigned long long *fallbacks,
                    const float bound, const float dead_zone, int *status,
                    float *__restrict__ trace) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kOffMisc);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kOffMisc + kNumBars * 8);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  int *counts = reinterpret_cast<int *>(tmem_slot + 2);  // loads issued, stages landed
  float *sb = reinterpret_cast<float *>(smem + kOffMisc + 256);  // b1, b2, b3
  auto bar = [&](int k) -> uint32_t { return smem_u32(bars + k); };

  // ---- weights (canonical layouts) and biases
  for (int q = tid; q < kTaps * 2 * kMlpHidden; q += kConvThreads) {
    const int tap = q / (2 * kMlpHidden), rem = q - tap * 2 * kMlpHidden;
    const int h = rem / kMlpHidden, n = rem - h * kMlpHidden;
    uint32_t w[4];
#pragma unroll
    for (int c = 0; c < 8; c += 2) {
      const int k0 = 8 * h + c;
      const __nv_bfloat16 *src = p.w1 + n * kMlpIn + kMlpMoments * tap + k0;
      const uint16_t lo = k0 < kMlpMoments ? __bfloat16_as_ushort(src[0]) : 0;
      const uint16_t hi = k0 + 1 < kMlpMoments ? __bfloat16_as_ushort(src[1]) : 0;
      w[c / 2] = (uint32_t)lo | ((uint32_t)hi << 16);
    }
    *reinterpret_cast<uint4 *>(smem + kOffW1 + tap * kTapBytes + h * 1024 + n * 16) =
        make_uint4(w[0], w[1], w[2], w[3]);
  }
  for (int c = tid; c < kMlpHidden * (kMlpHidden / 8); c += kConvThreads) {
    const int n = c / (kMlpHidden / 8), kb = c - n * (kMlpHidden / 8);
    *reinterpret_cast<uint4 *>(smem + kOffW2 + cm_offset(n, 8 * kb, kMlpHidden)) =
        *reinterpret_cast<const uint4 *>(p.w2 + n * kMlpHidden + 8 * kb);
  }
  for (int c = tid; c < kMlpOut * (kMlpHidden / 8); c += kConvThreads) {
    const int n = c / (kMlpHidden / 8), kb = c - n * (kMlpHidden / 8);
    *reinterpret_cast<uint4 *>(smem + kOffW3 + cm_offset(n, 8 * kb, kMlpHidden)) =
        *reinterpret_cast<const uint4 *>(p.w3 + n * kMlpHidden + 8 * kb);
  }
  for (int c = tid; c < 2 * kMlpHidden + kMlpOut; c += kConvThreads)
    sb[c] = c < kMlpHidden ? p.b1[c] : (c < 2 * kMlpHidden ? p.b2[c - kMlpHidden]
                                                           : p.b3[c - 2 * kMlpHidden]);
  if (tid == 0) {
    for (int k = 0; k < kNumBars; ++k)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar(k)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    *abort_flag = 0;
    counts[0] = counts[1] = 0;
  }
  if (warp == 1) {
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
  const uint32_t lim = wait_limit(status);
  const long long ntiles = g.n / kCRows;
  const uint32_t sw1 = smem_u32(smem + kOffW1), sw2 = smem_u32(smem + kOffW2);
  const uint32_t sw3 = smem_u32(smem + kOffW3), sa1 = smem_u32(smem + kOffA1);

  if (warp == 0) {
    // ---------------------------------------------------------- producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&xs_map))
                   : "memory");
      int issued = 0;
      for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        if (*abort_flag) break;
        const int s = issued % kStages, use = issued / kStages;
        if (!mbar_wait(bar(kBarEmpty + s), (use & 1) ^ 1, lim)) {
          *abort_flag = 1;
          break;
        }
        mbar_expect_tx(bar(kBarFull + s), kTxBytes);
        // tile -> (x0, y, z) in 32-bit arithmetic (the launcher keeps the
        // tile count below 2^31)
        const uint32_t t = (uint32_t)tile, tpr = (uint32_t)g.nx / kCRows;
        const uint32_t row = t / tpr;
        const int x0 = (int)(t - row * tpr) * kCRows;
        const int y = (int)(row % (uint32_t)g.ny), z = (int)(row / (uint32_t)g.ny);
#pragma unroll 1
        for (int r9 = 0; r9 < 9; ++r9) {
          const int dy = r9 % 3 - 1, dz = r9 / 3 - 1;
#pragma unroll
          for (int h = 0; h < 2; ++h)
            tma_load_4d(sa1 + s * kStageBytes + (2 * r9 + h) * kHalfPitch, &xs_map, 8 * h, x0,
                        y + dy + 1, z + dz + 1, bar(kBarFull + s));
        }
        ++issued;
      }
      counts[0] = issued;
    }
  } else if (warp == 1) {
    // ------------------------------------------------- layer-1 MMA issuer
    if (lane == 0) {
      int landed = 0;
      for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        if (*abort_flag) break;
        const int j = landed, s = j % kStages, gs = j % kGroups;
        if (!mbar_wait(bar(kBarFull + s), (j / kStages) & 1, lim)) {
          *abort_flag = 1;
          break;
        }
        ++landed;
        if (!mbar_wait(bar(kBarAcc1E + gs), ((j / kGroups) & 1) ^ 1, lim)) {
          *abort_flag = 1;
          break;
        }
        fence_after();
        // descriptors of tap 0; a tap adds its byte offset / 16 to the start
        // address field (no carry: shared addresses stay below 256 KB)
        const uint64_t a0 = sdesc(sa1 + s * kStageBytes, kHalfPitch, 128);
        const uint64_t b0 = sdesc(sw1, 1024, 128);
        const uint32_t d = tmem + 128 * gs;
#pragma unroll
        for (int tap = 0; tap < kTaps; ++tap) {
          const uint32_t aoff = 2 * (tap / 3) * kHalfPitch + (tap % 3) * 16;
          umma(d, a0 + (aoff >> 4), b0 + ((tap * kTapBytes) >> 4),
               idesc_bf16(kCRows, kMlpHidden), tap > 0);
        }
        umma_commit(bar(kBarEmpty + s));
        umma_commit(bar(kBarAcc1F + gs));
      }
      counts[1] = landed;
    }
  } else {
    // --------------------------------------------------- epilogue groups
    const int eg = (warp - 2) >> 2;             // group 0 .. kGroups - 1
    const int quarter = warp & 3;               // TMEM lanes 32 quarter .. (warp % 4 rule)
    const int r = 32 * quarter + lane;          // tile row
    const bool leader = warp == 2 + 4 * eg && lane == 0;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * quarter) << 16);
    unsigned char *a2 = smem + kOffA2 + eg * kA2Bytes;
    const uint32_t sa2 = smem_u32(a2);
    const uint32_t c1 = 128 * eg, c2 = 128 * eg + 64, c3 = c2;  // layer 1, 2, 3 columns
    uint32_t ph2 = 0, ph3 = 0;
    int j = eg;  // the block's tile index
    for (long long tile = blockIdx.x + (long long)eg * gridDim.x; tile < ntiles;
         tile += (long long)kGroups * gridDim.x, j += kGroups) {
      bool ok = mbar_wait(bar(kBarAcc1F + eg), (j / kGroups) & 1, lim);
      if (group_any(eg, !ok || *abort_flag)) {
        *abort_flag = 1;
        break;
      }
      fence_after();
      uint32_t v[32];
      float *trace_row = TRACE ? trace + ((long long)tile * kCRows + r) * kConvTrace : nullptr;
      // layer 1 epilogue (hidden row 1), releasing the accumulator once read
      load_acc32(lane_addr + c1, v);
      hidden_half<TRACE>(v, sb, 0, a2, r, trace_row);
      load_acc32(lane_addr + c1 + 32, v);
      fence_before();
      group_sync(eg);
      if (leader) mbar_arrive(bar(kBarAcc1E + eg));
      hidden_half<TRACE>(v, sb, 32, a2, r, trace_row);
      fence_async_smem();
      group_sync(eg);
      if (leader) {
        fence_after();
#pragma unroll
        for (int ks = 0; ks < kMlpHidden / 16; ++ks)
          umma(tmem + c2, sdesc(sa2 + 256 * ks, 128, (kMlpHidden / 8) * 128),
               sdesc(sw2 + 256 * ks, 128, (kMlpHidden / 8) * 128),
               idesc_bf16(kCRows, kMlpHidden), ks > 0);
        umma_commit(bar(kBarL2 + eg));
      }
      ok = mbar_wait(bar(kBarL2 + eg), ph2, lim);
      ph2 ^= 1;
      if (group_any(eg, !ok)) {
        *abort_flag = 1;
        break;
      }
      fence_after();
      // layer 2 epilogue (hidden row 2 over row 1, which layer 2 has read)
      load_acc32(lane_addr + c2, v);
      hidden_half<TRACE>(v, sb + kMlpHidden, 0, a2, r, TRACE ? trace_row + kMlpHidden : nullptr);
      load_acc32(lane_addr + c2 + 32, v);
      hidden_half<TRACE>(v, sb + kMlpHidden, 32, a2, r, TRACE ? trace_row + kMlpHidden : nullptr);
      fence_async_smem();
      fence_before();
      group_sync(eg);
      if (leader) {
        fence_after();
#pragma unroll
        for (int ks = 0; ks < kMlpHidden / 16; ++ks)
          umma(tmem + c3, sdesc(sa2 + 256 * ks, 128, (kMlpHidden / 8) * 128),
               sdesc(sw3 + 256 * ks, 128, (kMlpHidden / 8) * 128), idesc_bf16(kCRows, kMlpOut),
               ks > 0);
        umma_commit(bar(kBarL3 + eg));
      }
      ok = mbar_wait(bar(kBarL3 + eg), ph3, lim);
      ph3 ^= 1;
      if (group_any(eg, !ok)) {
        *abort_flag = 1;
        break;
      }
      fence_after();
      load_acc32(lane_addr + c3, v);
      fence_before();
      // the closure update of this row's cell with its 17 predictions
      const float *b3 = sb + 2 * kMlpHidden;
      float yk[kMlpOutUsed];
#pragma unroll
      for (int k = 0; k < kMlpOutUsed; ++k) yk[k] = __uint_as_float(v[k]) + b3[k];
      if (TRACE)
#pragma unroll
        for (int k = 0; k < kMlpOutUsed; ++k) trace_row[2 * kMlpHidden + k] = yk[k];
      const uint32_t t = (uint32_t)tile, tpr = (uint32_t)g.nx / kCRows;
      const uint32_t row = t / tpr;
      const int x = (int)(t - row * tpr) * kCRows + r;
      closure_update_cell<PARITY, IDX>(p, f, g, om1, x, (int)(row % (uint32_t)g.ny),
                                       (int)(row / (uint32_t)g.ny), yk, fallbacks, bound,
                                       dead_zone);
    }
  }

  __syncthreads();
  if (*abort_flag) {
    // copies and MMAs still in flight land before the memory goes away
    if (tid == 0) {
      atomicExch(status, 1);
      for (int k = counts[1]; k < counts[0]; ++k)
        mbar_wait(bar(kBarFull + k % kStages), (k / kStages) & 1);
    }
    const bool lead = warp >= 2 && ((warp - 2) & 3) == 0 && lane == 0;
    if ((warp == 1 && lane == 0) || lead) {
      const int d = warp == 1 ? 0 : 1 + ((warp - 2) >> 2);
      umma_commit(bar(kBarDrain + d));
      mbar_wait(bar(kBarDrain + d), 0);
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
}

// Feature source: standardised moments (BF16, 16 channels) of every cell of
// the periodically padded grid, from the logical populations of an FP32 store.
// The same moments and rounding as the features of lb_closure_features.
__global__ void __launch_bounds__(256)
    feature_source_kernel(MlpDevice p, const float *__restrict__ f, const Grid g, const int parity,
                          uint4 *__restrict__ xs) {
  const long long px = g.nx + 2, py = g.ny + 2, pz = g.nz + 2;
  const long long q = (long long)blockIdx.x * 256 + threadIdx.x;
  if (q >= px * py * pz) return;
  const int X = (int)(q % px);
  const long long t = q / px;
  const int Yp = (int)(t % py), Z = (int)(t / py);
  const int x = X == 0 ? g.nx - 1 : (X == g.nx + 1 ? 0 : X - 1);
  const int y = Yp == 0 ? g.ny - 1 : (Yp == g.ny + 1 ? 0 : Yp - 1);
  const int z = Z == 0 ? g.nz - 1 : (Z == g.nz + 1 ? 0 : Z - 1);
  float df[27];
  load_logical<27, 0>(f, g, parity, x, y, z, df);
  const Macro m = Lattice<27>::moments(df);
  const float v[kMlpMoments] = {m.drho, m.ux, m.uy, m.uz, m.pxx, m.pxy, m.pxz, m.pyy, m.pyz, m.pzz};
  uint32_t w[5];
#pragma unroll
  for (int k = 0; k < kMlpMoments; k += 2)
    w[k / 2] = pack_bf16((v[k] - p.in_mean[k]) * p.in_inv_std[k],
                         (v[k + 1] - p.in_mean[k + 1]) * p.in_inv_std[k + 1]);
  xs[2 * q] = make_uint4(w[0], w[1], w[2], w[3]);
  xs[2 * q + 1] = make_uint4(w[4], 0u, 0u, 0u);
}

}  // namespace

bool mlp_conv_supported(const Grid &g) { return g.nx % kCRows == 0 && g.walls == 0; }

size_t feature_source_bytes(const Grid &g) {
  return (size_t)(g.nx + 2) * (size_t)(g.ny + 2) * (size_t)(g.nz + 2) * 32;
}

cudaError_t make_feature_map(void *xs, const Grid &g, CUtensorMap *map) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    cudaError_t e =
        cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[4] = {16, (cuuint64_t)g.nx + 2, (cuuint64_t)g.ny + 2,
                              (cuuint64_t)g.nz + 2};
  const cuuint64_t strides[3] = {32, 32 * dims[1], 32 * dims[1] * dims[2]};
  const cuuint32_t box[4] = {8, (cuuint32_t)kCSpan, 1, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, xs, dims, strides, box,
                            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_feature_source(const MlpDevice &p, const float *f, const Grid &g, int parity,
                                  void *xs, cudaStream_t st) {
  const long long cells = (long long)(g.nx + 2) * (g.ny + 2) * (g.nz + 2);
  feature_source_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, st>>>(
      p, f, g, parity, static_cast<uint4 *>(xs));
  return cudaGetLastError();
}

cudaError_t launch_mlp_conv_step(const MlpDevice &p, const CUtensorMap &map, const Grid &g,
                                 float *f, float om1, int parity, unsigned long long *fallbacks,
                                 float bound, float dead_zone, int *status, int nblocks,
                                 cudaStream_t st, float *trace) {
  // 32-bit element offsets where every slot of the store is addressable so
  auto kern = trace ? (parity ? mlp_conv_kernel<1, long long, true>
                              : mlp_conv_kernel<0, long long, true>)
              : 27 * g.n < (1LL << 31) ? (parity ? mlp_conv_kernel<1, int> : mlp_conv_kernel<0, int>)
                                       : (parity ? mlp_conv_kernel<1, long long>
                                                 : mlp_conv_kernel<0, long long>);
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kConvSmem);
  if (e != cudaSuccess) return e;
  const long long tiles = g.n / kCRows;
  if (tiles >= (1LL << 31)) return cudaErrorInvalidValue;
  const int nb = (int)(tiles < nblocks ? tiles : nblocks);
  if (nb < 1) return cudaSuccess;
  kern<<<nb, kConvThreads, kConvSmem, st>>>(p, map, g, f, om1, fallbacks, bound, dead_zone,
                                            status, trace);
  return cudaGetLastError();
}

}  // namespace lbrr
