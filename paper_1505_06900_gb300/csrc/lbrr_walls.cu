// Collide-and-stream update with no-slip walls (Sec. 3.7, boundary
// conditions) on an AA-pattern store, for grids whose Grid::walls is set.
//
// The walls pass through the first and last node planes of the walled axes:
// boundary nodes lie on the walls and carry u_bc = 0. In either AA parity,
// population i of node x is unknown when x - xi_i lies beyond a wall plane
// (nothing streamed it in); a boundary node fills its unknown populations
// (wall_fill), takes rho and Pi^(1) from the filled set with u = 0
// (wall_macro), and relaxes to f0(rho, 0) + (1 - 1/tau) f1(Pi^(1)), which is
// the regularization formula followed by the collision for every model (at
// u = 0 the RR, order-2 regularized and BGK updates of a regularized state
// coincide). Post-collision populations whose destination x + xi_i lies
// beyond a wall plane are not stored. Off the walls the update is that of
// rr_step_kernel. Indices wrap periodically, so an unknown population is read
// from a valid (unrelated) location before it is replaced.
//
// One thread per node, blocks along x; bytes per update as in the periodic
// kernel. Any storage precision.
#include "lbrr_launch.h"

namespace lbrr {

constexpr int kWallThreads = 128;

template <int Q, int S, int MODEL, int PARITY>
__global__ void __launch_bounds__(kWallThreads)
    rr_step_walls_kernel(typename Storage<S>::T *__restrict__ f, const Grid g, const float om1) {
  using St = Storage<S>;
  using L = Lattice<Q>;
  constexpr int D = L::D;
  const int x = blockIdx.x * kWallThreads + threadIdx.x;
  if (x >= g.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const long long n = g.n;
  const uint32_t unknown = unknown_mask<Q>(g, x, y, z);
  float df[Q];

  const int xs[3] = {wrap_add(x, -1, g.nx), x, wrap_add(x, 1, g.nx)};
  const int ys[3] = {wrap_add(y, -1, g.ny), y, wrap_add(y, 1, g.ny)};
  int zs[3] = {0, 0, 0};
  if (D == 3) {
    zs[0] = wrap_add(z, -1, g.nz);
    zs[1] = z;
    zs[2] = wrap_add(z, 1, g.nz);
  }
  auto row = [&](int b, int c) -> long long { return ((long long)zs[c] * g.ny + ys[b]) * g.nx; };
  const long long cell = row(1, 1) + x;

  if (PARITY == 0) {
#pragma unroll
    for (int i = 0; i < Q; ++i) df[i] = St::template load<Q>(f + i * n + cell, i);
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int cx = vel_q<Q>(i, 0), cy = vel_q<Q>(i, 1);
      const int cz = (D == 3) ? vel_q<Q>(i, 2) : 0;
      df[i] = St::template load<Q>(f + (Q - 1 - i) * n + row(1 - cy, 1 - cz) + xs[1 - cx], i);
    }
  }
  if (unknown) {
    wall_fill<Q>(unknown, df);
    Macro m = L::moments(df);
    wall_macro(m);
    L::template synth<0>(m, om1, df);
  } else {
    const Macro m = L::moments(df);
    L::template synth<MODEL>(m, om1, df);
  }
  if (PARITY == 0) {
#pragma unroll
    for (int i = 0; i < Q; ++i) St::template store<Q>(f + (Q - 1 - i) * n + cell, i, df[i]);
  } else {
    const uint32_t outgoing = opposite_mask<Q>(unknown);  // destination beyond a wall
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if ((outgoing >> i) & 1u) continue;
      const int cx = vel_q<Q>(i, 0), cy = vel_q<Q>(i, 1);
      const int cz = (D == 3) ? vel_q<Q>(i, 2) : 0;
      St::template store<Q>(f + i * n + row(1 + cy, 1 + cz) + xs[1 + cx], i, df[i]);
    }
  }
}

template <int Q, int S, int MODEL>
static cudaError_t walls_t(void *f, const Grid &g, float om1, int parity, cudaStream_t st) {
  using T = typename Storage<S>::T;
  const dim3 grid((g.nx + kWallThreads - 1) / kWallThreads, g.ny, g.nz);
  if (parity == 0)
    rr_step_walls_kernel<Q, S, MODEL, 0><<<grid, kWallThreads, 0, st>>>(static_cast<T *>(f), g,
                                                                         om1);
  else
    rr_step_walls_kernel<Q, S, MODEL, 1><<<grid, kWallThreads, 0, st>>>(static_cast<T *>(f), g,
                                                                         om1);
  return cudaGetLastError();
}

template <int Q, int S>
static cudaError_t walls_m(int model, void *f, const Grid &g, float om1, int parity,
                           cudaStream_t st) {
  switch (model) {
    case 0: return walls_t<Q, S, 0>(f, g, om1, parity, st);
    case 1: return walls_t<Q, S, 1>(f, g, om1, parity, st);
    default: return walls_t<Q, S, 2>(f, g, om1, parity, st);
  }
}

template <int Q>
static cudaError_t walls_s(int storage, int model, void *f, const Grid &g, float om1, int parity,
                           cudaStream_t st) {
  switch (storage) {
    case 0: return walls_m<Q, 0>(model, f, g, om1, parity, st);
    case 1: return walls_m<Q, 1>(model, f, g, om1, parity, st);
    default: return walls_m<Q, 2>(model, f, g, om1, parity, st);
  }
}

cudaError_t launch_step_walls(int q, int storage, int model, void *f, const Grid &g, float om1,
                              int parity, cudaStream_t st) {
  if (q == 9) return walls_s<9>(storage, model, f, g, om1, parity, st);
  if (q == 19) return walls_s<19>(storage, model, f, g, om1, parity, st);
  return walls_s<27>(storage, model, f, g, om1, parity, st);
}

}  // namespace lbrr
