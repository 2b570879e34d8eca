// Collide-and-stream kernel for the 16-bit population stores (FP16 / BF16,
// holding g = (f - w) / w), tiled through shared memory.
//
// With 2-byte populations a one-thread-per-cell kernel issues one memory
// instruction per 2 bytes and keeps too few bytes in flight to saturate HBM.
// Here a block owns one row segment of kTileX cells at (y, z). It stages, for
// each of the Q slots, the 16-byte chunks of the row that slot is read from
// (cp.async, 16 bytes per copy), including an 8-value halo on both sides for
// the x +- 1 shifts of the odd AA update; each thread then collides its cell
// from shared memory, writes the post-collision values back into the tile at
// their streamed positions, and the block stores every whole 16-byte chunk it
// owns with one vector store (edge values that share a chunk with a
// neighbouring segment are stored one by one).
//
// AA pattern as in lbrr_step.cu: parity 0 reads and writes the cell's own
// slots (population i into slot opp(i)); parity 1 reads slot opp(i) of
// x - xi_i and writes slot i of x + xi_i. Slot s is therefore read from and
// written to the same row (y + cy_s, z + cz_s) in an odd update. A location
// outside the block's cells may be read as halo while its owner rewrites it;
// the value is never used. Requires nx to be a multiple of kTileX.
//
// The per-cell arithmetic runs on g with the weights folded into the
// separable moment passes (ratios 1 : 4 : 1) and divided out of the
// synthesis, all in float32.
#include "lbrr_launch.h"

namespace lbrr {

constexpr int kTileX = 128;                    // cells per block (one per thread)
constexpr int kHalo = 8;                       // one 16-byte chunk of halo per side
constexpr int kRowLen = kTileX + 2 * kHalo;    // staged values per slot
constexpr int kChunk = 8;                      // 16-bit values per 16-byte chunk

template <int S>
struct Half;
template <>
struct Half<1> {
  __device__ __forceinline__ static float to_f(__half v) { return __half2float(v); }
  __device__ __forceinline__ static __half from_f(float v) { return __float2half_rn(v); }
};
template <>
struct Half<2> {
  __device__ __forceinline__ static float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
  __device__ __forceinline__ static __nv_bfloat16 from_f(float v) {
    return __float2bfloat16_rn(v);
  }
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <int Q, int S, int MODEL, int PARITY>
__global__ void __launch_bounds__(kTileX)
    rr_step_tiled16_kernel(typename Storage<S>::T *__restrict__ f, const Grid g, const float om1) {
  using T = typename Storage<S>::T;
  using L = Lattice<Q>;
  constexpr int D = L::D;
  constexpr int kInner = kTileX / kChunk;  // chunks of the block's own cells per slot
  __shared__ __align__(16) T tile[Q][kRowLen];

  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * kTileX;
  const int y = blockIdx.y, z = blockIdx.z;
  const long long n = g.n;

  // offset of the first value of slot s in row (y + cy_s, z + cz_s) (odd) or
  // (y, z) (even), computed once per block
  __shared__ long long srow[Q];
  if (tid < Q) {
    int yy = y, zz = z;
    if (PARITY) {
      yy = wrap_add(y, vel(tid, 1), g.ny);
      zz = D == 3 ? wrap_add(z, vel(tid, 2), g.nz) : 0;
    }
    srow[tid] = (long long)tid * n + ((long long)zz * g.ny + yy) * g.nx;
  }
  __syncthreads();
  auto slot_row = [&](int s) -> T * { return f + srow[s]; };

  // ---- stage the block's segment of every slot (16-byte async copies) ...
  for (int p = tid; p < Q * kInner; p += kTileX) {
    const int s = p / kInner, k = p - s * kInner;
    cp_async16(&tile[s][kHalo + kChunk * k], slot_row(s) + x0 + kChunk * k);
  }
  // ... and, for the odd update, one halo chunk on each side (periodic in x)
  if (PARITY) {
    for (int p = tid; p < 2 * Q; p += kTileX) {
      const int s = p >> 1, side = p & 1;
      const int xg = side ? (x0 + kTileX == g.nx ? 0 : x0 + kTileX)
                          : (x0 == 0 ? g.nx - kChunk : x0 - kChunk);
      cp_async16(&tile[s][side ? kHalo + kTileX : 0], slot_row(s) + xg);
    }
  }
  cp_async_wait_all();
  __syncthreads();

  // ---- collide the thread's cell
  float v[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int s = PARITY ? Q - 1 - i : i;
    v[i] = Half<S>::to_f(tile[s][kHalo + tid - (PARITY ? vel(i, 0) : 0)]);
  }
  __syncthreads();  // every input is in registers before outputs overwrite the tile
  const Macro m = L::template moments<true>(v);
  L::template synth<MODEL, true>(m, om1, v);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int s = PARITY ? i : Q - 1 - i;
    tile[s][kHalo + tid + (PARITY ? vel(i, 0) : 0)] = Half<S>::from_f(v[i]);
  }
  __syncthreads();

  // ---- store the values this block owns. Slot s of an odd update owns the
  // tile positions [kHalo + cx_s, kHalo + kTileX + cx_s): whole 16-byte chunks
  // go out as vector stores, the 8 values per shifted slot that share a chunk
  // with a neighbouring segment one by one.
  for (int p = tid; p < Q * kInner; p += kTileX) {
    const int s = p / kInner, k = p - s * kInner;
    if (PARITY) {
      const int cx = vel(s, 0);
      if ((cx > 0 && k == 0) || (cx < 0 && k == kInner - 1)) continue;
    }
    *reinterpret_cast<uint4 *>(slot_row(s) + x0 + kChunk * k) =
        *reinterpret_cast<const uint4 *>(&tile[s][kHalo + kChunk * k]);
  }
  if (PARITY) {
    for (int p = tid; p < Q * kChunk; p += kTileX) {
      const int s = p / kChunk, t = p - s * kChunk;
      const int cx = vel(s, 0);
      if (cx == 0) continue;
      // cx = +1: positions kHalo+1 .. kHalo+7 and kHalo+kTileX
      // cx = -1: positions kHalo-1 and kHalo+kTileX-8 .. kHalo+kTileX-2
      const int j = cx > 0 ? (t < kChunk - 1 ? kHalo + 1 + t : kHalo + kTileX)
                           : (t == 0 ? kHalo - 1 : kHalo + kTileX - kChunk - 1 + t);
      int xg = x0 - kHalo + j;
      xg = xg < 0 ? xg + g.nx : (xg >= g.nx ? xg - g.nx : xg);
      slot_row(s)[xg] = tile[s][j];
    }
  }
}

template <int Q, int S, int MODEL>
static cudaError_t tiled_t(void *f, const Grid &g, float om1, int parity, cudaStream_t st) {
  using T = typename Storage<S>::T;
  const dim3 grid(g.nx / kTileX, g.ny, g.nz);
  if (parity == 0)
    rr_step_tiled16_kernel<Q, S, MODEL, 0><<<grid, kTileX, 0, st>>>(static_cast<T *>(f), g, om1);
  else
    rr_step_tiled16_kernel<Q, S, MODEL, 1><<<grid, kTileX, 0, st>>>(static_cast<T *>(f), g, om1);
  return cudaGetLastError();
}

bool tiled16_supported(const Grid &g) { return g.nx % kTileX == 0; }

template <int Q, int S>
static cudaError_t tiled_m(int model, void *f, const Grid &g, float om1, int parity,
                           cudaStream_t st) {
  switch (model) {
    case 0: return tiled_t<Q, S, 0>(f, g, om1, parity, st);
    case 1: return tiled_t<Q, S, 1>(f, g, om1, parity, st);
    default: return tiled_t<Q, S, 2>(f, g, om1, parity, st);
  }
}

cudaError_t launch_step_tiled16(int q, int storage, int model, void *f, const Grid &g, float om1,
                                int parity, cudaStream_t st) {
  if (q == 9)
    return storage == 1 ? tiled_m<9, 1>(model, f, g, om1, parity, st)
                        : tiled_m<9, 2>(model, f, g, om1, parity, st);
  return storage == 1 ? tiled_m<27, 1>(model, f, g, om1, parity, st)
                      : tiled_m<27, 2>(model, f, g, om1, parity, st);
}

}  // namespace lbrr
