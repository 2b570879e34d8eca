// Even (in-place) collide-and-stream update of the 16-bit population stores
// (FP16 / BF16, holding g = (f - w) / w) with direct coalesced accesses.
//
// AA pattern as in lbrr_step.cu: the even update reads the cell's own slots
// and writes post-collision population i into slot opp(i) of the same cell,
// so no access is shifted. Each thread owns two neighbouring cells (x0,
// x0 + 1), x0 even, and moves every slot of both as one aligned 32-bit word:
// a warp reads or writes one whole 128-byte line per slot, as the FP32
// kernel does, with no shared-memory staging and no block barrier. The
// collision runs in packed FP32x2 arithmetic (lbrr_pair.cuh). The odd update,
// whose x-shifted slots straddle words, stays with the staged segment kernel
// (lbrr_step16.cu). Requires nx % 64 == 0 (whole warps per row); blocks of 128
// threads cover 256 cells of one row.
#include "lbrr_launch.h"
#include "lbrr_pair.cuh"

namespace lbrr {

constexpr int kPairThreads = 128;
constexpr int kPairCells = 2 * kPairThreads;

template <int S>
__device__ __forceinline__ float2 unpack2(uint32_t w) {
  using T2 = typename Half<S>::T2;
  return Half<S>::to_f2(*reinterpret_cast<const T2 *>(&w));
}
template <int S>
__device__ __forceinline__ uint32_t pack2(float2 v) {
  using T2 = typename Half<S>::T2;
  const T2 h = Half<S>::from_f2(v);
  return *reinterpret_cast<const uint32_t *>(&h);
}

template <int Q, int S, int MODEL>
__global__ void __launch_bounds__(kPairThreads)
    rr_step_pair16_even_kernel(uint32_t *__restrict__ w, const Grid g, const float om1) {
  const int x0 = blockIdx.x * kPairCells + 2 * threadIdx.x;
  if (x0 >= g.nx) return;
  const long long nw = g.n >> 1;  // words per slot (n is even)
  const long long cw = (((long long)blockIdx.z * g.ny + blockIdx.y) * g.nx + x0) >> 1;
  float2 v[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) v[i] = unpack2<S>(w[i * nw + cw]);
  pair::collide<Q, MODEL>(v, om1);
  // The stores go to the addresses of the loads (slot Q - 1 - i of the same
  // words). Passing the offset through an empty asm makes the compiler
  // compute them anew here instead of holding all Q of them in registers
  // across the collision: 72 instead of 124 registers a thread for D3Q27 RR.
  long long cw_out = cw;
  asm volatile("" : "+l"(cw_out));
#pragma unroll
  for (int i = 0; i < Q; ++i) w[(Q - 1 - i) * nw + cw_out] = pack2<S>(v[i]);
}

template <int Q, int S, int MODEL>
static cudaError_t pair_t(void *f, const Grid &g, float om1, cudaStream_t st) {
  const dim3 grid((g.nx + kPairCells - 1) / kPairCells, g.ny, g.nz);
  rr_step_pair16_even_kernel<Q, S, MODEL>
      <<<grid, kPairThreads, 0, st>>>(static_cast<uint32_t *>(f), g, om1);
  return cudaGetLastError();
}

template <int Q, int S>
static cudaError_t pair_m(int model, void *f, const Grid &g, float om1, cudaStream_t st) {
  switch (model) {
    case 0: return pair_t<Q, S, 0>(f, g, om1, st);
    case 1: return pair_t<Q, S, 1>(f, g, om1, st);
    default: return pair_t<Q, S, 2>(f, g, om1, st);
  }
}

bool pair16_even_supported(const Grid &g) { return g.nx % 64 == 0; }

cudaError_t launch_step_pair16_even(int q, int storage, int model, void *f, const Grid &g,
                                    float om1, cudaStream_t st) {
  if (q == 9)
    return storage == 1 ? pair_m<9, 1>(model, f, g, om1, st) : pair_m<9, 2>(model, f, g, om1, st);
  if (q == 19)
    return storage == 1 ? pair_m<19, 1>(model, f, g, om1, st)
                        : pair_m<19, 2>(model, f, g, om1, st);
  return storage == 1 ? pair_m<27, 1>(model, f, g, om1, st) : pair_m<27, 2>(model, f, g, om1, st);
}

}  // namespace lbrr
