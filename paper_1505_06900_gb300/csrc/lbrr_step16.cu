// Collide-and-stream kernel for the 16-bit population stores (FP16 / BF16,
// holding g = (f - w) / w), tiled through shared memory.
//
// With 2-byte populations a one-thread-per-cell kernel issues one memory
// instruction per 2 bytes and keeps too few bytes in flight to saturate HBM.
// Here a block owns one row segment of TX cells at (y, z) (TX = 256 where nx
// allows, else 128; TX / 2 threads). It stages, for
// each of the Q slots, the 16-byte chunks of the row that slot is read from
// (cp.async, 16 bytes per copy), including an 8-value halo on both sides for
// the x +- 1 shifts of the odd AA update; each thread then collides two
// neighbouring cells from shared memory in packed FP32x2 arithmetic
// (lbrr_pair.cuh), writes the post-collision values back into the tile at
// their streamed positions, and the block stores every whole 16-byte chunk it
// owns with one vector store (edge values that share a chunk with a
// neighbouring segment are stored one by one). Unshifted slots move between
// shared memory and registers as packed 32-bit pairs.
//
// AA pattern as in lbrr_step.cu: parity 0 reads and writes the cell's own
// slots (population i into slot opp(i)); parity 1 reads slot opp(i) of
// x - xi_i and writes slot i of x + xi_i. Slot s is therefore read from and
// written to the same row (y + cy_s, z + cz_s) in an odd update. A location
// outside the block's cells may be read as halo while its owner rewrites it;
// the value is never used. Requires nx to be a multiple of TX. The library
// launches the odd form only (see tiled_tx below).
#include <algorithm>

#include "lbrr_launch.h"
#include "lbrr_pair.cuh"

namespace lbrr {

constexpr int kTileX = 128;                    // shortest row segment (cells per block)
constexpr int kHalo = 8;                       // one 16-byte chunk of halo per side
constexpr int kChunk = 8;                      // 16-bit values per 16-byte chunk

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Slots of the Q-velocity lattice with cx = -1 (and, mirrored, cx = +1):
// shifted_slot<Q>(k, pos) is the k-th slot with cx = +1 (pos) or -1, of the
// shifted_slots<Q>() of each sign.
template <int Q>
__host__ __device__ constexpr int shifted_slots() { return Q == 19 ? 5 : Q / 3; }
template <int Q>
__host__ __device__ constexpr int shifted_slot(int k, bool pos) {
  // D2Q9 / D3Q27: 3k (cx = -1), 3k + 2 (cx = +1); D3Q19: 1, 5, 8, 11, 15 and
  // 3, 7, 10, 13, 17
  return Q == 19 ? (pos ? 3 : 1) + 3 * k + (k >= 1) + (k >= 4) : 3 * k + (pos ? 2 : 0);
}
template <int Q>
constexpr bool shifted_slots_ok() {
  int np = 0, nm = 0;
  for (int i = 0; i < Q; ++i) {
    np += vel_q<Q>(i, 0) == 1;
    nm += vel_q<Q>(i, 0) == -1;
  }
  if (np != shifted_slots<Q>() || nm != shifted_slots<Q>()) return false;
  for (int k = 0; k < shifted_slots<Q>(); ++k)
    if (vel_q<Q>(shifted_slot<Q>(k, true), 0) != 1 || vel_q<Q>(shifted_slot<Q>(k, false), 0) != -1)
      return false;
  return true;
}
static_assert(shifted_slots_ok<9>() && shifted_slots_ok<19>() && shifted_slots_ok<27>(),
              "shifted-slot tables");

template <int Q, int S, int MODEL, int PARITY, int TX>
__global__ void __launch_bounds__(TX / 2)
    rr_step_tiled16_kernel(typename Storage<S>::T *__restrict__ f, const Grid g, const float om1) {
  using T = typename Storage<S>::T;
  using T2 = typename Half<S>::T2;
  constexpr int D = Lattice<Q>::D;
  constexpr int kThreads = TX / 2;         // two cells per thread
  constexpr int kInner = TX / kChunk;      // chunks of the block's own cells per slot
  __shared__ __align__(16) T tile[Q][TX + 2 * kHalo];

  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX;
  const int y = blockIdx.y, z = blockIdx.z;
  const long long n = g.n;

  // offset of the first value of slot s in row (y + cy_s, z + cz_s) (odd) or
  // (y, z) (even), computed once per block
  __shared__ long long srow[Q];
  if (tid < Q) {
    int yy = y, zz = z;
    if (PARITY) {
      yy = wrap_add(y, vel_q<Q>(tid, 1), g.ny);
      zz = D == 3 ? wrap_add(z, vel_q<Q>(tid, 2), g.nz) : 0;
    }
    srow[tid] = (long long)tid * n + ((long long)zz * g.ny + yy) * g.nx;
  }
  __syncthreads();
  auto slot_row = [&](int s) -> T * { return f + srow[s]; };

  // Chunk loops: thread tid moves chunk k = tid % kInner of the slots
  // s = tid / kInner + j * kSlotStep, j = 0, 1, ...
  constexpr int kSlotStep = kThreads / kInner;
  constexpr int kSlotIters = (Q + kSlotStep - 1) / kSlotStep;
  const int kc = tid % kInner, s0 = tid / kInner;

  // ---- stage the block's segment of every slot (16-byte async copies) ...
#pragma unroll
  for (int j = 0; j < kSlotIters; ++j) {
    const int s = s0 + j * kSlotStep;
    if (s < Q) cp_async16(&tile[s][kHalo + kChunk * kc], slot_row(s) + x0 + kChunk * kc);
  }
  // ... and, for the odd update, one halo chunk on each side (periodic in x)
  if (PARITY) {
    static_assert(2 * Q <= kThreads, "one halo chunk per thread");
    if (tid < 2 * Q) {
      const int s = tid >> 1, side = tid & 1;
      const int xg = side ? (x0 + TX == g.nx ? 0 : x0 + TX)
                          : (x0 == 0 ? g.nx - kChunk : x0 - kChunk);
      cp_async16(&tile[s][side ? kHalo + TX : 0], slot_row(s) + xg);
    }
  }
  cp_async_wait_all();
  __syncthreads();

  // ---- collide the thread's two cells (x0 + 2 tid, x0 + 2 tid + 1)
  const int c0 = kHalo + 2 * tid;
  float2 v[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int s = PARITY ? Q - 1 - i : i;
    const int sh = PARITY ? vel_q<Q>(i, 0) : 0;
    const T *p = &tile[s][c0 - sh];
    if (sh == 0)
      v[i] = Half<S>::to_f2(*reinterpret_cast<const T2 *>(p));
    else
      v[i] = make_float2(Half<S>::to_f(p[0]), Half<S>::to_f(p[1]));
  }
  __syncthreads();  // every input is in registers before outputs overwrite the tile
  pair::collide<Q, MODEL>(v, om1);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int s = PARITY ? i : Q - 1 - i;
    const int sh = PARITY ? vel_q<Q>(i, 0) : 0;
    T *p = &tile[s][c0 + sh];
    if (sh == 0) {
      *reinterpret_cast<T2 *>(p) = Half<S>::from_f2(v[i]);
    } else {
      p[0] = Half<S>::from_f(v[i].x);
      p[1] = Half<S>::from_f(v[i].y);
    }
  }
  __syncthreads();

  // ---- store the values this block owns. Slot s of an odd update owns the
  // tile positions [kHalo + cx_s, kHalo + TX + cx_s): whole 16-byte chunks
  // go out as vector stores, the 8 values per shifted slot that share a chunk
  // with a neighbouring segment one by one.
  // Bit masks of the slots with cx = +1 and cx = -1.
  constexpr uint32_t kPosMask = vel_mask<Q>(0, 1);
  constexpr uint32_t kNegMask = vel_mask<Q>(0, -1);
  const uint32_t skip = !PARITY ? 0u
                                : (kc == 0 ? kPosMask : 0u) | (kc == kInner - 1 ? kNegMask : 0u);
#pragma unroll
  for (int j = 0; j < kSlotIters; ++j) {
    const int s = s0 + j * kSlotStep;
    if (s < Q && !((skip >> s) & 1u))
      *reinterpret_cast<uint4 *>(slot_row(s) + x0 + kChunk * kc) =
          *reinterpret_cast<const uint4 *>(&tile[s][kHalo + kChunk * kc]);
  }
  if (PARITY) {
    // 8 values of each shifted slot: item p -> shifted slot m = p / 8 (the
    // (m / 2)-th slot with cx = -1 for even m, with cx = +1 for odd m), value t
    constexpr int kEdgeItems = 2 * shifted_slots<Q>() * kChunk;
#pragma unroll
    for (int p = tid; p < kEdgeItems; p += kThreads) {
      const int m = p / kChunk, t = p % kChunk;
      const bool pos = m & 1;
      const int s = shifted_slot<Q>(m >> 1, pos);
      // cx = +1: positions kHalo+1 .. kHalo+7 and kHalo+TX
      // cx = -1: positions kHalo-1 and kHalo+TX-8 .. kHalo+TX-2
      const int j = pos ? (t < kChunk - 1 ? kHalo + 1 + t : kHalo + TX)
                        : (t == 0 ? kHalo - 1 : kHalo + TX - kChunk - 1 + t);
      int xg = x0 - kHalo + j;
      xg = xg < 0 ? xg + g.nx : (xg >= g.nx ? xg - g.nx : xg);
      slot_row(s)[xg] = tile[s][j];
    }
  }
}

// ------------------------------------------------------------------------
// Row kernel: a persistent block owns whole x-rows (y, z), one after the
// other. For each row it copies the Q slot rows (the row each slot is read
// from: (y, z) in an even update, (y + cy_s, z + cz_s) in an odd one) into
// shared memory with one 1-D bulk copy per slot (cp.async.bulk, completion on
// an mbarrier), collides two cells per thread in place, and writes the Q rows
// back with one bulk store per slot. With the whole row in shared memory the
// periodic x-shifts wrap inside it: no halo, and every output position is
// owned by the block that computes it. kRowBufs row buffers let the copies
// of the next kRowDist rows run during the current row's collision, without
// waiting for the stores of the row before. Each (slot, row) pair is
// read and written by exactly one row of the update, so rows never race.
// Requires nx % 16 == 0 (16-byte rows), nx >= 64 (a thread per slot) and
// nx / 2 threads per block (nx <= 1024 for D3Q27 and D3Q19, 2048 for D2Q9).

constexpr uint32_t kRowWaitLimit = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity,
                                          uint32_t limit = kRowWaitLimit) {
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
// global -> shared bulk copy, completing `bytes` on the mbarrier
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes,
                                          uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}
// shared -> global bulk copy in this thread's bulk group
__device__ __forceinline__ void bulk_store(void *dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst),
               "r"(src), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}
// this thread's bulk stores are complete
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
}

// largest row (cells) of the row kernel: D3Q27 and D3Q19 keep <= 512 threads
// so that a thread has the registers of a pair without spilling
template <int Q>
constexpr int row16_max_nx() { return Q == 9 ? 2048 : 1024; }

// Row buffers in shared memory and how many rows ahead the copies run: the
// buffer refilled for row k + kRowDist was last stored kRowBufs - kRowDist
// rows before, so with kRowDist <= kRowBufs - 2 its store has had a whole
// row's time to read it (kRowDist = kRowBufs - 1 waits for the newest store).
constexpr int kRowBufs = 3;
constexpr int kRowDist = 1;
static_assert(kRowDist >= 1 && kRowDist <= kRowBufs - 1, "at least one row in flight");

// this thread's bulk stores except the newest n have finished reading shared memory
template <int N>
__device__ __forceinline__ void bulk_wait_read_but() {
  asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(N) : "memory");
}

template <int Q, int S, int MODEL, int PARITY>
__global__ void __launch_bounds__(row16_max_nx<Q>() / 2)
    rr_step_row16_kernel(typename Storage<S>::T *__restrict__ f, const Grid g, const float om1,
                         int *status) {
  using T = typename Storage<S>::T;
  using T2 = typename Half<S>::T2;
  constexpr int D = Lattice<Q>::D;
  extern __shared__ __align__(128) unsigned char smem_row[];
  const int nx = g.nx;
  const int rows = g.ny * g.nz;
  T *const buf0 = reinterpret_cast<T *>(smem_row);
  const size_t buf_elems = (size_t)Q * nx;
  uint64_t *const mbar =
      reinterpret_cast<uint64_t *>(smem_row + kRowBufs * buf_elems * sizeof(T));
  const int tid = threadIdx.x;
  const uint32_t row_bytes = (uint32_t)(nx * sizeof(T));
  // main-loop wait limit: status[1] when positive (host test of the timeout
  // path), else kRowWaitLimit; the cleanup waits always use kRowWaitLimit
  const uint32_t lim = status[1] > 0 ? (uint32_t)status[1] : kRowWaitLimit;

  if (tid == 0) {
#pragma unroll
    for (int k = 0; k < kRowBufs; ++k) mbar_init(smem_u32(&mbar[k]));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();

  // first element of slot s's row for the update of row r
  auto slot_row = [&](int s, int r) -> T * {
    int y = r % g.ny, z = r / g.ny;
    if (PARITY) {
      y = wrap_add(y, vel_q<Q>(s, 1), g.ny);
      z = D == 3 ? wrap_add(z, vel_q<Q>(s, 2), g.nz) : 0;
    }
    return f + (long long)s * g.n + ((long long)z * g.ny + y) * nx;
  };
  // warp 0 copies the Q slot rows of row r into buffer b (thread s: slot s),
  // after this thread's store from that buffer has read it
  auto issue_load = [&](int r, int b) {
    if (tid < 32) {
      if (tid == 0) mbar_expect_tx(smem_u32(&mbar[b]), (uint32_t)Q * row_bytes);
      __syncwarp();
      if (tid < Q) {
        bulk_wait_read_but<kRowBufs - kRowDist - 1>();
        bulk_load(smem_u32(buf0 + b * buf_elems + (size_t)tid * nx), slot_row(tid, r), row_bytes,
                  smem_u32(&mbar[b]));
      }
    }
  };

  // the thread's cells x = 2 tid, 2 tid + 1 and their periodic x - 1, x + 2
  const int xa = 2 * tid;
  const int xm = tid == 0 ? nx - 1 : xa - 1;
  const int xp = xa + 2 == nx ? 0 : xa + 2;

  uint32_t phases = 0;  // bit k: parity of the next completion of mbar[k]
  int b = 0;            // buffer of the current row
  bool ok = true;
  // prologue: rows blockIdx.x + j * gridDim.x, j < kRowDist
#pragma unroll
  for (int j = 0; j < kRowDist; ++j) {
    const long long r = blockIdx.x + (long long)j * gridDim.x;
    if (r < rows) issue_load((int)r, j);
  }
  int r = blockIdx.x;
  for (; r < rows; r += gridDim.x) {
    const long long rn = r + (long long)kRowDist * gridDim.x;
    int bn = b + kRowDist;
    bn = bn >= kRowBufs ? bn - kRowBufs : bn;
    if (rn < rows) issue_load((int)rn, bn);
    const bool got = mbar_wait(smem_u32(&mbar[b]), (phases >> b) & 1u, lim);
    if (__syncthreads_or(!got)) {
      ok = false;
      break;
    }
    phases ^= 1u << b;
    T *const t = buf0 + b * buf_elems;

    float2 v[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int s = PARITY ? Q - 1 - i : i;
      const int sh = PARITY ? vel_q<Q>(i, 0) : 0;  // read at x - sh
      const T *p = t + (size_t)s * nx;
      if (sh == 0)
        v[i] = Half<S>::to_f2(*reinterpret_cast<const T2 *>(p + xa));
      else if (sh > 0)
        v[i] = make_float2(Half<S>::to_f(p[xm]), Half<S>::to_f(p[xa]));
      else
        v[i] = make_float2(Half<S>::to_f(p[xa + 1]), Half<S>::to_f(p[xp]));
    }
    __syncthreads();  // every input is in registers before outputs overwrite the row
    pair::collide<Q, MODEL>(v, om1);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int s = PARITY ? i : Q - 1 - i;
      const int sh = PARITY ? vel_q<Q>(i, 0) : 0;  // write at x + sh
      T *p = t + (size_t)s * nx;
      if (sh == 0) {
        *reinterpret_cast<T2 *>(p + xa) = Half<S>::from_f2(v[i]);
      } else if (sh > 0) {
        p[xa + 1] = Half<S>::from_f(v[i].x);
        p[xp] = Half<S>::from_f(v[i].y);
      } else {
        p[xm] = Half<S>::from_f(v[i].x);
        p[xa] = Half<S>::from_f(v[i].y);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // visible to the bulk copies
    __syncthreads();
    if (tid < Q) bulk_store(slot_row(tid, r), smem_u32(t + (size_t)tid * nx), row_bytes);
    b = b + 1 == kRowBufs ? 0 : b + 1;
  }
  if (!ok) {
    // record the timeout; let the copies in flight (rows r .. r + kRowDist)
    // land before the block exits
    if (tid == 0) atomicExch(status, 1);
    int bb = b;
    for (int j = 0; j <= kRowDist; ++j) {
      if (r + (long long)j * gridDim.x < rows) mbar_wait(smem_u32(&mbar[bb]), (phases >> bb) & 1u);
      bb = bb + 1 == kRowBufs ? 0 : bb + 1;
    }
  }
  if (tid < Q) bulk_wait_all();
}

template <int Q, int S, int MODEL, int PARITY>
static cudaError_t row_launch(void *f, const Grid &g, float om1, int *status, cudaStream_t st,
                              bool &launched) {
  using T = typename Storage<S>::T;
  auto kern = rr_step_row16_kernel<Q, S, MODEL, PARITY>;
  const size_t smem = kRowBufs * (size_t)Q * g.nx * sizeof(T) + kRowBufs * sizeof(uint64_t);
  const int threads = g.nx / 2;
  if (smem > 48 * 1024) {  // opt in to more than the default dynamic shared memory
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) {
      cudaGetLastError();
      launched = false;
      return cudaSuccess;
    }
  }
  int per_sm = 0, dev = 0, sms = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) {
    launched = false;
    return cudaSuccess;
  }
  const long long rows = (long long)g.ny * g.nz;
  const int blocks = (int)std::min<long long>(rows, (long long)per_sm * sms);
  kern<<<blocks, threads, smem, st>>>(static_cast<T *>(f), g, om1, status);
  launched = true;
  return cudaGetLastError();
}

template <int Q, int S>
static cudaError_t row_m(int model, void *f, const Grid &g, float om1, int parity, int *status,
                         cudaStream_t st, bool &launched) {
  switch (model * 2 + parity) {
    case 0: return row_launch<Q, S, 0, 0>(f, g, om1, status, st, launched);
    case 1: return row_launch<Q, S, 0, 1>(f, g, om1, status, st, launched);
    case 2: return row_launch<Q, S, 1, 0>(f, g, om1, status, st, launched);
    case 3: return row_launch<Q, S, 1, 1>(f, g, om1, status, st, launched);
    case 4: return row_launch<Q, S, 2, 0>(f, g, om1, status, st, launched);
    default: return row_launch<Q, S, 2, 1>(f, g, om1, status, st, launched);
  }
}

cudaError_t launch_step_row16(int q, int storage, int model, void *f, const Grid &g, float om1,
                              int parity, int *status, cudaStream_t st, bool &launched) {
  launched = false;
  if (g.nx % 16 != 0 || g.nx < 64 || !status) return cudaSuccess;
  if (g.nx > (q == 9 ? row16_max_nx<9>() : row16_max_nx<27>())) return cudaSuccess;
  if (q == 9)
    return storage == 1 ? row_m<9, 1>(model, f, g, om1, parity, status, st, launched)
                        : row_m<9, 2>(model, f, g, om1, parity, status, st, launched);
  if (q == 19)
    return storage == 1 ? row_m<19, 1>(model, f, g, om1, parity, status, st, launched)
                        : row_m<19, 2>(model, f, g, om1, parity, status, st, launched);
  return storage == 1 ? row_m<27, 1>(model, f, g, om1, parity, status, st, launched)
                      : row_m<27, 2>(model, f, g, om1, parity, status, st, launched);
}

// Only the odd form is launched: every row length this kernel takes
// (nx % 128 == 0) has its even update in the direct kernel of lbrr_pair16.cu.
template <int Q, int S, int MODEL, int TX>
static cudaError_t tiled_tx(void *f, const Grid &g, float om1, cudaStream_t st) {
  using T = typename Storage<S>::T;
  const dim3 grid(g.nx / TX, g.ny, g.nz);
  rr_step_tiled16_kernel<Q, S, MODEL, 1, TX><<<grid, TX / 2, 0, st>>>(static_cast<T *>(f), g, om1);
  return cudaGetLastError();
}

template <int Q, int S, int MODEL>
static cudaError_t tiled_t(void *f, const Grid &g, float om1, cudaStream_t st) {
  if (g.nx % 256 == 0) return tiled_tx<Q, S, MODEL, 256>(f, g, om1, st);
  return tiled_tx<Q, S, MODEL, 128>(f, g, om1, st);
}

bool tiled16_supported(const Grid &g) { return g.nx % kTileX == 0; }

template <int Q, int S>
static cudaError_t tiled_m(int model, void *f, const Grid &g, float om1, cudaStream_t st) {
  switch (model) {
    case 0: return tiled_t<Q, S, 0>(f, g, om1, st);
    case 1: return tiled_t<Q, S, 1>(f, g, om1, st);
    default: return tiled_t<Q, S, 2>(f, g, om1, st);
  }
}

cudaError_t launch_step_tiled16_odd(int q, int storage, int model, void *f, const Grid &g,
                                    float om1, cudaStream_t st) {
  if (q == 9)
    return storage == 1 ? tiled_m<9, 1>(model, f, g, om1, st)
                        : tiled_m<9, 2>(model, f, g, om1, st);
  if (q == 19)
    return storage == 1 ? tiled_m<19, 1>(model, f, g, om1, st)
                        : tiled_m<19, 2>(model, f, g, om1, st);
  return storage == 1 ? tiled_m<27, 1>(model, f, g, om1, st)
                      : tiled_m<27, 2>(model, f, g, om1, st);
}

}  // namespace lbrr
