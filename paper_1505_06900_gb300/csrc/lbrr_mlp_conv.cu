// Closure-network forward pass fused with the closure update, for grids whose
// rows are whole 128-cell tiles, fed by the tensor memory accelerator (TMA)
// and pipelined across tiles.
//
// Layer 1 of the network is a 3x3x3 convolution of the standardised moment
// field: its 270 inputs for a cell are the 10 moments of the 27 cells around
// it. A feature-source tensor holds those moments once per position of the
// grid with a one-cell periodic halo (X = x + 1, Y = y + 1, Z = z + 1), BF16,
// split in two halves of 8 channels, each half laid out [Z][Y][X][8] with
// rows padded to nx + 8 positions:
//   half 0: moments 0..7 (rho - 1, ux, uy, uz, Pi xx, xy, xz, yy) at X;
//   half 1: moments 8, 9 (Pi yz, zz) at X - 1, X and X + 1, then two ones
//           (the constant input through which layer 1 adds its bias).
// For a tile of 128 cells x0 .. x0 + 127 of row (y, z) the producer copies,
// per half and per z plane Z = z .. z + 2, the 3 neighbour rows Y = y .. y + 2
// over the positions X = x0 .. x0 + 135 in one TMA tile load whose rows are
// 128-byte chunks of 8 positions. In shared memory each neighbour row is then
// [136 positions][16 bytes]: the canonical K-major layout without swizzle
// (8-row groups 128 bytes apart) with position X = x0 + r at row r, so that
// a cell's neighbour at dx is row m + dx + 1 of its tile row m. Layer 1 is
// 18 MMAs (M 128, N 64, K 16, K = 288 in all), two per neighbour row, each
// reading two 8-channel K blocks through the leading byte offset of its
// descriptor: (half 0 at dx = -1, half 0 at dx = 0), 16 bytes apart, and
// (half 0 at dx = +1, half 1 at dx = 0), the latter holding moments 8 and 9
// of all three dx. The weight operand of each MMA is W1's 16 matching
// columns; at the centre row the two constant inputs meet b1 split into
// BF16 b_hi + b_lo (b1 - b_hi - b_lo is below 2^-18 |b1|).
//
// One persistent block per SM, nineteen warps:
//   warp 0      TMA producer: per tile 2 tile loads (halves) for each of the 3 z
//               planes of one of 2 stages; a plane has its own full / empty
//               barriers, so the next tile's first plane loads while the MMAs
//               still read the later planes of this one
//   warps 1, 2  layer-1 MMA issuers of alternate tiles (warp 1 owns the TMEM),
//               so that one waits for its next plane while the other issues
//   warps 3-18  four epilogue groups of four warps taking every fourth tile;
//               thread = TMEM lane = tile row. When a group starts a tile,
//               each thread sends the 27 populations its cell's update reads
//               to shared memory (cp.async). The group then reads its layer-1
//               accumulator (bias included), applies tanh and stores the BF16
//               hidden row back into tensor memory, where layer 2 takes it
//               as its A operand (issued by the group); the same for layer
//               2 and layer 3. With the 17 standardised outputs of its row
//               and the staged populations each thread performs the closure
//               update of its cell in the population store
//               (closure_update_cell_df): the step of the learned closure is
//               fused into the network.
// Group g owns TMEM columns 128 g .. 128 g + 127: the first 64 take its
// layer-1 accumulator and then the hidden rows h1 and h2 (32 columns), and
// go back to the layer-1 MMAs once layer 3 has read h2; the other 64 take
// its layer 2 and then layer 3.
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
#include "lbrr_act.cuh"
#include "lbrr_tc.cuh"

namespace lbrr {

namespace {

using namespace tc;

constexpr int kCRows = 128;                         // cells per tile
constexpr int kChunk = 8;                           // positions per 128-byte TMA row
constexpr int kRowPos = 136;                        // staged positions x0 - 1 .. x0 + 134
constexpr int kPadPos = 8;                          // padded row: nx + 8 positions
constexpr uint32_t kRowBytes = kRowPos * 16;        // one neighbour row of one half
constexpr uint32_t kHalfBytes = 9 * kRowBytes;      // the 9 neighbour rows of one half
constexpr uint32_t kStageBytes = 2 * kHalfBytes;
constexpr int kStages = 2;
constexpr int kParts = 3;                           // z planes of a stage, each with its barriers
constexpr int kPartRows = 9 / kParts;               // neighbour rows of a part (per half)
constexpr uint32_t kTxPart = 2 * kPartRows * kRowBytes;  // bytes a part receives
constexpr int kMmas1 = 18;                          // layer-1 MMAs, K = 16 each
constexpr uint32_t kW1Bytes = 2 * kMlpHidden * 16;  // W1 block of one layer-1 MMA
static_assert(kRowPos % kChunk == 0 && kRowPos >= kCRows + 2, "staged row covers the taps");
static_assert(kPadPos % kChunk == 0 && kPadPos >= kRowPos - kCRows, "last box inside the row");
constexpr uint32_t kPopBytes = 27 * kCRows * 4;    // populations of one tile, [27][128]
constexpr int kGroups = 4;                          // epilogue groups
constexpr int kIssuers = 2;                         // layer-1 MMA warps
constexpr int kEpiWarp0 = 1 + kIssuers;             // first warp of the epilogue groups
constexpr int kConvThreads = 32 * (kEpiWarp0 + 4 * kGroups);
constexpr uint32_t kTmemCols = 512;

constexpr uint32_t kSmW1 = 0;
constexpr uint32_t kSmW2 = kSmW1 + kMmas1 * kW1Bytes;
constexpr uint32_t kSmW3 = kSmW2 + kMlpHidden * kMlpHidden * 2;
constexpr uint32_t kOffA1 = kSmW3 + kMlpOut * kMlpHidden * 2;
constexpr uint32_t kOffPop = kOffA1 + kStages * kStageBytes;
constexpr uint32_t kOffMisc = kOffPop + kGroups * kPopBytes;
constexpr uint32_t kOffBias = 512;                   // biases, after barriers and counters
// b1 (not read: layer 1 takes its bias through the constant inputs), b2,
// b3, then the 17 output scales
constexpr uint32_t kConvSmem = kOffMisc + kOffBias + 4 * (2 * kMlpHidden + kMlpOut + kMlpOutUsed);
static_assert(kOffA1 % 128 == 0 && kStageBytes % 128 == 0 && kHalfBytes % 128 == 0,
              "TMA destinations are 128-byte aligned");
static_assert(kConvSmem <= 232448, "fits the shared memory of one block");

// mbarriers in the misc area
enum : int {
  kBarFull = 0,                       // [stages x parts] part loaded (TMA transaction bytes)
  kBarEmpty = kBarFull + kStages * kParts,  // [stages x parts] part read by the layer-1 MMAs
  kBarAcc1F = kBarEmpty + kStages * kParts,  // [groups] layer-1 accumulator ready (commit)
  kBarAcc1E = kBarAcc1F + kGroups,    // [groups] layer-1 accumulator read by its group
  kBarL2 = kBarAcc1E + kGroups,       // [groups] layer 2 done
  kBarL3 = kBarL2 + kGroups,          // [groups] layer 3 done
  kBarDrain = kBarL3 + kGroups,       // [issuers + groups] drain of each MMA issuer after an abort
  kNumBars = kBarDrain + kIssuers + kGroups
};
static_assert(kNumBars * 8 + 8 + 4 * (1 + kIssuers) <= kOffBias,
              "barriers, TMEM slot, abort flag and counters before the biases");

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes)
               : "memory");
}
// 5-D tiled TMA load (coordinates innermost first), completing on mbar
__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, int c3, int c4, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
      "r"(mbar)
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

// tanh(acc + bias) of 32 accumulator columns c0 .. c0 + 31 (in v; without
// BIAS the accumulator holds the bias already), rounded to BF16 and packed
// two to a column into the 16 TMEM columns at taddr of this thread's lane
// (the row of the next layer's A operand); with TRACE also the FP32 values
// into trace_row[c0 ..].
template <bool TRACE = false, bool BIAS = true>
__device__ __forceinline__ void hidden_tmem(const uint32_t (&v)[32], const float *bias, int c0,
                                            uint32_t taddr, float *trace_row = nullptr) {
  uint32_t q[16];
#pragma unroll
  for (int k = 0; k < 32; k += 4) {
    float z0 = __uint_as_float(v[k]), z1 = __uint_as_float(v[k + 1]);
    float z2 = __uint_as_float(v[k + 2]), z3 = __uint_as_float(v[k + 3]);
    if (BIAS) {
      const float4 b = *reinterpret_cast<const float4 *>(bias + c0 + k);
      z0 += b.x;
      z1 += b.y;
      z2 += b.z;
      z3 += b.w;
    }
    const float h0 = tanh_approx(z0), h1 = tanh_approx(z1);
    const float h2 = tanh_approx(z2), h3 = tanh_approx(z3);
    if (TRACE) {
      trace_row[c0 + k] = h0;
      trace_row[c0 + k + 1] = h1;
      trace_row[c0 + k + 2] = h2;
      trace_row[c0 + k + 3] = h3;
    }
    q[k / 2] = pack_bf16(h0, h1);
    q[k / 2 + 1] = pack_bf16(h2, h3);
  }
  tmem_st16(taddr, q);
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
  int *counts = reinterpret_cast<int *>(tmem_slot + 2);  // parts issued, seen per issuer
  float *sb = reinterpret_cast<float *>(smem + kOffMisc + kOffBias);  // b1, b2, b3
  auto bar = [&](int k) -> uint32_t { return smem_u32(bars + k); };

  // ---- weights (canonical layouts) and biases
  // layer-1 MMA q = 2 r9 + kind of neighbour row r9 = (dy + 1) + 3 (dz + 1),
  // K block h: feature 10 nb + ch of neighbour nb = (dx + 1) + 3 r9, as the
  // A operand's blocks hold them (see above)
  for (int q = tid; q < kMmas1 * 2 * kMlpHidden; q += kConvThreads) {
    const int mq = q / (2 * kMlpHidden), rem = q - mq * 2 * kMlpHidden;
    const int h = rem / kMlpHidden, n = rem - h * kMlpHidden;
    const int r9 = mq >> 1, kind = mq & 1;
    uint16_t w[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      int nb, ch;
      if (kind == 0 || h == 0) {  // moments 0..7 of dx = -1 / 0 (kind 0), dx = +1 (kind 1)
        nb = (kind == 0 ? h : 2) + 3 * r9;
        ch = k;
      } else {  // moments 8, 9 of dx = -1, 0, +1, then the constant inputs
        nb = k < 6 ? (k >> 1) + 3 * r9 : -1;
        ch = 8 + (k & 1);
      }
      w[k] = nb >= 0 ? __bfloat16_as_ushort(p.w1[n * kMlpIn + kMlpMoments * nb + ch]) : 0;
    }
    if (kind == 1 && h == 1 && r9 == 4) {  // b1 = b_hi + b_lo on the constant inputs
      const __nv_bfloat16 hi = __float2bfloat16_rn(p.b1[n]);
      w[6] = __bfloat16_as_ushort(hi);
      w[7] = __bfloat16_as_ushort(__float2bfloat16_rn(p.b1[n] - __bfloat162float(hi)));
    }
    *reinterpret_cast<uint4 *>(smem + kSmW1 + mq * kW1Bytes + h * 1024 + n * 16) =
        make_uint4(w[0] | ((uint32_t)w[1] << 16), w[2] | ((uint32_t)w[3] << 16),
                   w[4] | ((uint32_t)w[5] << 16), w[6] | ((uint32_t)w[7] << 16));
  }
  for (int c = tid; c < kMlpHidden * (kMlpHidden / 8); c += kConvThreads) {
    const int n = c / (kMlpHidden / 8), kb = c - n * (kMlpHidden / 8);
    *reinterpret_cast<uint4 *>(smem + kSmW2 + cm_offset(n, 8 * kb, kMlpHidden)) =
        *reinterpret_cast<const uint4 *>(p.w2 + n * kMlpHidden + 8 * kb);
  }
  for (int c = tid; c < kMlpOut * (kMlpHidden / 8); c += kConvThreads) {
    const int n = c / (kMlpHidden / 8), kb = c - n * (kMlpHidden / 8);
    *reinterpret_cast<uint4 *>(smem + kSmW3 + cm_offset(n, 8 * kb, kMlpHidden)) =
        *reinterpret_cast<const uint4 *>(p.w3 + n * kMlpHidden + 8 * kb);
  }
  for (int c = tid; c < 2 * kMlpHidden + kMlpOut + kMlpOutUsed; c += kConvThreads)
    sb[c] = c < kMlpHidden ? p.b1[c]
            : c < 2 * kMlpHidden ? p.b2[c - kMlpHidden]
            : c < 2 * kMlpHidden + kMlpOut ? p.b3[c - 2 * kMlpHidden]
                                           : p.out_scale[c - 2 * kMlpHidden - kMlpOut];
  if (tid == 0) {
    for (int k = 0; k < kNumBars; ++k)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar(k)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    *abort_flag = 0;
    for (int k = 0; k <= kIssuers; ++k) counts[k] = 0;
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
  const uint32_t sw1 = smem_u32(smem + kSmW1), sw2 = smem_u32(smem + kSmW2);
  const uint32_t sw3 = smem_u32(smem + kSmW3), sa1 = smem_u32(smem + kOffA1);

  if (warp == 0) {
    // ---------------------------------------------------------- producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&xs_map))
                   : "memory");
      int issued = 0;  // parts
      bool stop = false;
      for (long long tile = blockIdx.x; tile < ntiles && !stop; tile += gridDim.x) {
        const int j = issued / kParts, s = j % kStages, use = j / kStages;
        // tile -> (x0, y, z) in 32-bit arithmetic (the launcher keeps the
        // tile count below 2^31)
        const uint32_t t = (uint32_t)tile, tpr = (uint32_t)g.nx / kCRows;
        const uint32_t row = t / tpr;
        const int x0 = (int)(t - row * tpr) * kCRows;
        const int y = (int)(row % (uint32_t)g.ny), z = (int)(row / (uint32_t)g.ny);
        // part k: the z plane Z = z + k (padded), rows Y = y .. y + 2, chunks from X = x0
        for (int k = 0; k < kParts; ++k) {
          const int b = s * kParts + k;
          if (*abort_flag || !mbar_wait(bar(kBarEmpty + b), (use & 1) ^ 1, lim)) {
            *abort_flag = 1;
            stop = true;
            break;
          }
          mbar_expect_tx(bar(kBarFull + b), kTxPart);
#pragma unroll
          for (int h = 0; h < 2; ++h)
            tma_load_5d(sa1 + s * kStageBytes + h * kHalfBytes + k * kPartRows * kRowBytes,
                        &xs_map, 0, x0 / kChunk, y, z + k * (3 / kParts), h, bar(kBarFull + b));
          ++issued;
        }
      }
      counts[0] = issued;
    }
  } else if (warp <= kIssuers) {
    // ------------------------------------------------ layer-1 MMA issuers:
    // warp 1 + i takes the tiles j = i mod kIssuers (stage j mod kStages)
    if (lane == 0) {
      const int iw = warp - 1;
      int landed = 0, nt = 0;  // parts seen, tiles started
      bool stop = false;
      for (long long tile = blockIdx.x + (long long)iw * gridDim.x; tile < ntiles && !stop;
           tile += (long long)kIssuers * gridDim.x, ++nt) {
        const int j = iw + kIssuers * nt, s = j % kStages, gs = j % kGroups;
        if (*abort_flag || !mbar_wait(bar(kBarAcc1E + gs), ((j / kGroups) & 1) ^ 1, lim)) {
          *abort_flag = 1;
          break;
        }
        // descriptors of neighbour row 0; a row adds its byte offset / 16 to
        // the start address field (no carry: shared addresses stay below
        // 256 KB). aP: rows m, m + 1 of half 0 (dx = -1, 0); aQ: row m + 2 of
        // half 0 (dx = +1) and row m + 1 of half 1 (moments 8, 9 of all dx).
        const uint32_t st = sa1 + s * kStageBytes;
        const uint64_t aP = sdesc(st, 16, 128);
        const uint64_t aQ = sdesc(st + 32, kHalfBytes - 16, 128);
        const uint64_t b0 = sdesc(sw1, 1024, 128);
        const uint32_t d = tmem + 128 * gs;
#pragma unroll
        for (int k = 0; k < kParts; ++k) {
          const int b = s * kParts + k;
          if (!mbar_wait(bar(kBarFull + b), (j / kStages) & 1, lim)) {
            *abort_flag = 1;
            stop = true;
            break;
          }
          ++landed;
          fence_after();
#pragma unroll
          for (int r9 = k * kPartRows; r9 < (k + 1) * kPartRows; ++r9) {
            const uint32_t ro = (r9 * kRowBytes) >> 4;
            umma(d, aP + ro, b0 + ((2 * r9 * kW1Bytes) >> 4), idesc_bf16(kCRows, kMlpHidden),
                 r9 > 0);
            umma(d, aQ + ro, b0 + (((2 * r9 + 1) * kW1Bytes) >> 4),
                 idesc_bf16(kCRows, kMlpHidden), 1);
          }
          umma_commit(bar(kBarEmpty + b));  // the part may be refilled once these are done
        }
        if (!stop) umma_commit(bar(kBarAcc1F + gs));
      }
      counts[1 + iw] = landed;
    }
  } else if (warp >= kEpiWarp0) {
    // --------------------------------------------------- epilogue groups
    const int eg = (warp - kEpiWarp0) >> 2;     // group 0 .. kGroups - 1
    const int quarter = warp & 3;               // TMEM lanes 32 quarter .. (warp % 4 rule)
    const int r = 32 * quarter + lane;          // tile row
    const bool leader = warp == kEpiWarp0 + 4 * eg && lane == 0;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * quarter) << 16);
    const float *pop = reinterpret_cast<const float *>(smem + kOffPop + eg * kPopBytes) + r;
    const uint32_t spop = smem_u32(pop);
    // columns: c1 the layer-1 accumulator, then the BF16 rows h1 and h2 (A
    // operands of layers 2 and 3) in its first 32 columns; c2 layer 2, then 3
    const uint32_t c1 = 128 * eg, c2 = 128 * eg + 64, c3 = c2;
    const uint32_t tpr = (uint32_t)g.nx / kCRows;
    uint32_t ph2 = 0, ph3 = 0;
    int j = eg;  // the block's tile index
    for (long long tile = blockIdx.x + (long long)eg * gridDim.x; tile < ntiles;
         tile += (long long)kGroups * gridDim.x, j += kGroups) {
      // this row's cell; its 27 populations go to shared memory while the
      // network runs (each cell reads only locations no other cell touches)
      const uint32_t t = (uint32_t)tile, row = t / tpr;
      const int x = (int)(t - row * tpr) * kCRows + r;
      const int y = (int)(row % (uint32_t)g.ny), z = (int)(row / (uint32_t)g.ny);
#pragma unroll
      for (int i = 0; i < 27; ++i)
        cp_async4(spop + i * kCRows * 4, f + closure_read_offset<PARITY, IDX>(g, x, y, z, i));
      cp_async_commit();
      bool ok = mbar_wait(bar(kBarAcc1F + eg), (j / kGroups) & 1, lim);
      if (group_any(eg, !ok || *abort_flag)) {
        *abort_flag = 1;
        break;
      }
      fence_after();
      uint32_t v[32];
      float *trace_row = TRACE ? trace + ((long long)tile * kCRows + r) * kConvTrace : nullptr;
      // layer 1 epilogue: h1 over the accumulator columns already read
      load_acc32(lane_addr + c1, v);
      hidden_tmem<TRACE, false>(v, sb, 0, lane_addr + c1, trace_row);
      load_acc32(lane_addr + c1 + 32, v);
      hidden_tmem<TRACE, false>(v, sb, 32, lane_addr + c1 + 16, trace_row);
      tmem_wait_st();
      fence_before();
      group_sync(eg);
      if (leader) {
        fence_after();
#pragma unroll
        for (int ks = 0; ks < kMlpHidden / 16; ++ks)
          umma_ts(tmem + c2, tmem + c1 + 8 * ks,
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
      // layer 2 epilogue: h2 over h1, which layer 2 has read
      load_acc32(lane_addr + c2, v);
      hidden_tmem<TRACE>(v, sb + kMlpHidden, 0, lane_addr + c1,
                         TRACE ? trace_row + kMlpHidden : nullptr);
      load_acc32(lane_addr + c2 + 32, v);
      hidden_tmem<TRACE>(v, sb + kMlpHidden, 32, lane_addr + c1 + 16,
                         TRACE ? trace_row + kMlpHidden : nullptr);
      tmem_wait_st();
      fence_before();
      group_sync(eg);
      if (leader) {
        fence_after();
#pragma unroll
        for (int ks = 0; ks < kMlpHidden / 16; ++ks)
          umma_ts(tmem + c3, tmem + c1 + 8 * ks,
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
      // layer 3 has read h2: the first 64 columns go back to the layer-1 MMAs
      if (leader) mbar_arrive(bar(kBarAcc1E + eg));
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
      cp_async_wait_all();
      float df[27];
#pragma unroll
      for (int i = 0; i < 27; ++i) df[i] = pop[i * kCRows];
      closure_update_cell_df<PARITY, IDX>(sb + 2 * kMlpHidden + kMlpOut, f, g, om1, x, y, z, df,
                                          yk, fallbacks, bound, dead_zone);
    }
    cp_async_wait_all();  // no copy into shared memory outlives the block
  }

  __syncthreads();
  if (*abort_flag) {
    // copies and MMAs still in flight land before the memory goes away
    if (tid == 0) {
      atomicExch(status, 1);
      // the parts no issuer has seen land (issuer i saw the first counts[1 + i]
      // parts of its tiles; a part of a stage holds at most one unseen load)
      for (int q = 0; q < counts[0]; ++q) {
        const int j = q / kParts, k = q % kParts, i = j % kIssuers;
        if (kParts * (j / kIssuers) + k >= counts[1 + i])
          mbar_wait(bar(kBarFull + (j % kStages) * kParts + k), (j / kStages) & 1);
      }
    }
    const bool lead = warp >= kEpiWarp0 && ((warp - kEpiWarp0) & 3) == 0 && lane == 0;
    if ((warp >= 1 && warp <= kIssuers && lane == 0) || lead) {
      const int d = warp <= kIssuers ? warp - 1 : kIssuers + ((warp - kEpiWarp0) >> 2);
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

// Feature source: standardised moments (BF16) of every position of the
// periodically padded grid, from the logical populations of an FP32 store,
// in the two halves described at the top of this file. The same moments and
// rounding as the features of lb_closure_features. A block of 256 threads
// computes 256 consecutive positions (x fastest) and writes the 254 inner
// ones, so that half 1 takes moments 8 and 9 of the neighbours at X - 1 and
// X + 1 from shared memory (for X = 0 and X = nx + 1, whose half 1 no tile
// reads, they come from the neighbouring rows).
constexpr int kFsThreads = 256, kFsOut = kFsThreads - 2;

__global__ void __launch_bounds__(kFsThreads)
    feature_source_kernel(MlpDevice p, const float *__restrict__ f, const Grid g, const int parity,
                          uint4 *__restrict__ xs) {
  __shared__ uint32_t s89[kFsThreads];
  const long long px = g.nx + 2, py = g.ny + 2, pz = g.nz + 2, total = px * py * pz;
  const long long q = (long long)blockIdx.x * kFsOut + threadIdx.x - 1;
  const bool valid = q >= 0 && q < total;
  uint32_t w[5] = {0u, 0u, 0u, 0u, 0u};
  long long row = 0;
  int X = 0;
  if (valid) {
    X = (int)(q % px);
    row = q / px;
    const int Yp = (int)(row % py), Z = (int)(row / py);
    const int x = X == 0 ? g.nx - 1 : (X == g.nx + 1 ? 0 : X - 1);
    const int y = Yp == 0 ? g.ny - 1 : (Yp == g.ny + 1 ? 0 : Yp - 1);
    const int z = Z == 0 ? g.nz - 1 : (Z == g.nz + 1 ? 0 : Z - 1);
    float df[27];
    load_logical<27, 0>(f, g, parity, x, y, z, df);
    const Macro m = Lattice<27>::moments(df);
    const float v[kMlpMoments] = {m.drho, m.ux,  m.uy,  m.uz,  m.pxx,
                                  m.pxy,  m.pxz, m.pyy, m.pyz, m.pzz};
#pragma unroll
    for (int k = 0; k < kMlpMoments; k += 2)
      w[k / 2] = pack_bf16((v[k] - p.in_mean[k]) * p.in_inv_std[k],
                           (v[k + 1] - p.in_mean[k + 1]) * p.in_inv_std[k + 1]);
  }
  s89[threadIdx.x] = w[4];
  __syncthreads();
  if (valid && threadIdx.x >= 1 && threadIdx.x <= kFsOut) {
    const long long o = row * (g.nx + kPadPos) + X;
    xs[o] = make_uint4(w[0], w[1], w[2], w[3]);
    xs[(long long)pz * py * (g.nx + kPadPos) + o] =
        make_uint4(s89[threadIdx.x - 1], w[4], s89[threadIdx.x + 1], 0x3F803F80u);  // 1.0, 1.0
  }
}

// The feature source in the channels-last form of lb_closure_step_trace:
// out[position][16], channels 0..9 the moments, 10..15 zero.
__global__ void __launch_bounds__(256)
    export_features_kernel(const uint4 *__restrict__ xs, const Grid g, uint4 *__restrict__ out) {
  const long long px = g.nx + 2, py = g.ny + 2, pz = g.nz + 2;
  const long long q = (long long)blockIdx.x * 256 + threadIdx.x;
  if (q >= px * py * pz) return;
  const long long o = (q / px) * (g.nx + kPadPos) + q % px;
  out[2 * q] = xs[o];
  out[2 * q + 1] = make_uint4(xs[pz * py * (g.nx + kPadPos) + o].y, 0u, 0u, 0u);
}

}  // namespace

bool mlp_conv_supported(const Grid &g) { return g.nx % kCRows == 0 && g.walls == 0; }

size_t feature_source_bytes(const Grid &g) {
  return 2 * (size_t)(g.nx + kPadPos) * (size_t)(g.ny + 2) * (size_t)(g.nz + 2) * 16;
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
  // [half][Z][Y][chunk][8 positions x 8 channels]
  const cuuint64_t rowb = (cuuint64_t)(g.nx + kPadPos) * 16;
  const cuuint64_t dims[5] = {8 * kChunk, (cuuint64_t)(g.nx + kPadPos) / kChunk,
                              (cuuint64_t)g.ny + 2, (cuuint64_t)g.nz + 2, 2};
  const cuuint64_t strides[4] = {16 * kChunk, rowb, rowb * dims[2], rowb * dims[2] * dims[3]};
  const cuuint32_t box[5] = {8 * kChunk, kRowPos / kChunk, 3, 3 / kParts, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, xs, dims, strides, box,
                            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_feature_source(const MlpDevice &p, const float *f, const Grid &g, int parity,
                                  void *xs, cudaStream_t st) {
  const long long cells = (long long)(g.nx + 2) * (g.ny + 2) * (g.nz + 2);
  feature_source_kernel<<<(unsigned)((cells + kFsOut - 1) / kFsOut), kFsThreads, 0, st>>>(
      p, f, g, parity, static_cast<uint4 *>(xs));
  return cudaGetLastError();
}

cudaError_t launch_export_features(const void *xs, const Grid &g, void *out, cudaStream_t st) {
  const long long cells = (long long)(g.nx + 2) * (g.ny + 2) * (g.nz + 2);
  export_features_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, st>>>(
      static_cast<const uint4 *>(xs), g, static_cast<uint4 *>(out));
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
