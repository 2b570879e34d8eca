// Fused collide-and-stream kernel of the recursive-regularized BGK scheme
// (arXiv:1505.06900, Sec. 3.5, eq_discr_bgk_reg) on an AA-pattern store.
//
// AA pattern: one population buffer, updated in place. With the store in
// natural order (parity 0), population i of cell x sits in slot i of x. An
// even update reads the cell's own slots, collides and writes post-collision
// population i into slot opp(i) of the same cell (streaming deferred). An odd
// update gathers population i of cell x from slot opp(i) of x - xi_i (where
// the previous update left it), collides and scatters population i into slot
// i of x + xi_i, which restores natural order. Each cell of an odd update
// reads exactly the locations it writes, so the in-place update is race-free.
//
// One thread per cell; a block covers a contiguous run of x in one (y, z)
// row, so every population slot is read and written by coalesced 4-byte (or
// 2-byte) accesses; the x +- 1 neighbours of the odd update shift a warp's
// window by one element, which costs one extra sector per access in L1/L2 but
// no extra DRAM traffic. The periodic wrap is folded into the index
// computation. Bytes per cell update: 2 Q sizeof(storage).
#include "lbrr_launch.h"

namespace lbrr {

constexpr int kStepThreads = 128;

template <int Q, int S, int MODEL, int PARITY>
__global__ void __launch_bounds__(kStepThreads)
    rr_step_kernel(typename Storage<S>::T *__restrict__ f, const Grid g, const float om1) {
  using St = Storage<S>;
  using L = Lattice<Q>;
  constexpr int D = L::D;
  const int x = blockIdx.x * kStepThreads + threadIdx.x;
  if (x >= g.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const long long n = g.n;
  float df[Q];

  if (PARITY == 0) {
    const long long cell = ((long long)z * g.ny + y) * g.nx + x;
#pragma unroll
    for (int i = 0; i < Q; ++i) df[i] = St::template load<Q>(f + i * n + cell, i);
    const Macro m = L::moments(df);
    L::template synth<MODEL>(m, om1, df);
#pragma unroll
    for (int i = 0; i < Q; ++i) St::template store<Q>(f + (Q - 1 - i) * n + cell, i, df[i]);
  } else {
    const int xs[3] = {wrap_add(x, -1, g.nx), x, wrap_add(x, 1, g.nx)};
    const int ys[3] = {wrap_add(y, -1, g.ny), y, wrap_add(y, 1, g.ny)};
    int zs[3] = {0, 0, 0};
    if (D == 3) {
      zs[0] = wrap_add(z, -1, g.nz);
      zs[1] = z;
      zs[2] = wrap_add(z, 1, g.nz);
    }
    // row(b, c): start of row y = ys[b], z = zs[c]
    auto row = [&](int b, int c) -> long long {
      return ((long long)zs[c] * g.ny + ys[b]) * g.nx;
    };
    // gather: population i of x lives in slot opp(i) of x - xi_i
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int cx = vel_q<Q>(i, 0), cy = vel_q<Q>(i, 1);
      const int cz = (D == 3) ? vel_q<Q>(i, 2) : 0;
      const long long src = row(1 - cy, 1 - cz) + xs[1 - cx];
      df[i] = St::template load<Q>(f + (Q - 1 - i) * n + src, i);
    }
    const Macro m = L::moments(df);
    L::template synth<MODEL>(m, om1, df);
    // scatter: population i goes to slot i of x + xi_i
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int cx = vel_q<Q>(i, 0), cy = vel_q<Q>(i, 1);
      const int cz = (D == 3) ? vel_q<Q>(i, 2) : 0;
      const long long dst = row(1 + cy, 1 + cz) + xs[1 + cx];
      St::template store<Q>(f + i * n + dst, i, df[i]);
    }
  }
}

template <int Q, int S, int MODEL>
static cudaError_t step_t(void *f, const Grid &g, float om1, int parity, cudaStream_t st) {
  using T = typename Storage<S>::T;
  const dim3 block(kStepThreads);
  const dim3 grid((g.nx + kStepThreads - 1) / kStepThreads, g.ny, g.nz);
  if (parity == 0)
    rr_step_kernel<Q, S, MODEL, 0><<<grid, block, 0, st>>>(static_cast<T *>(f), g, om1);
  else
    rr_step_kernel<Q, S, MODEL, 1><<<grid, block, 0, st>>>(static_cast<T *>(f), g, om1);
  return cudaGetLastError();
}

template <int Q, int S>
static cudaError_t step_m(int model, void *f, const Grid &g, float om1, int parity,
                          cudaStream_t st) {
  switch (model) {
    case 0: return step_t<Q, S, 0>(f, g, om1, parity, st);
    case 1: return step_t<Q, S, 1>(f, g, om1, parity, st);
    default: return step_t<Q, S, 2>(f, g, om1, parity, st);
  }
}

template <int Q>
static cudaError_t step_s(int storage, int model, void *f, const Grid &g, float om1, int parity,
                          cudaStream_t st) {
  switch (storage) {
    case 0: return step_m<Q, 0>(model, f, g, om1, parity, st);
    case 1: return step_m<Q, 1>(model, f, g, om1, parity, st);
    default: return step_m<Q, 2>(model, f, g, om1, parity, st);
  }
}

cudaError_t launch_step_cell(int q, int storage, int model, void *f, const Grid &g, float om1,
                             int parity, cudaStream_t st) {
  if (q == 9) return step_s<9>(storage, model, f, g, om1, parity, st);
  if (q == 19) return step_s<19>(storage, model, f, g, om1, parity, st);
  return step_s<27>(storage, model, f, g, om1, parity, st);
}

}  // namespace lbrr
