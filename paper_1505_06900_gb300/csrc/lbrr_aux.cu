// Initialisation, moment extraction, population copies and the FP64
// diagnostics reductions of the RR lattice Boltzmann library.
#include <type_traits>

#include "lbrr_launch.h"

namespace lbrr {

constexpr int kAuxThreads = 128;

// ------------------------------------------------------------------ init --
// f = f0(rho, u) [+ f1 with a1^(2) = -2 cs2 rho tau S]: the constitutive
// relation of Sec. 3.3 in lattice units, with tau the scheme's tau-bar; the
// higher orders of f1 follow from the recursion inside synth (om1 = 1).
template <int Q, int S, int MODEL>
__global__ void __launch_bounds__(kAuxThreads)
    init_kernel(typename Storage<S>::T *__restrict__ f, const Grid g,
                const float *__restrict__ rho, const float *__restrict__ u, const float tau,
                const int mode) {
  using L = Lattice<Q>;
  constexpr int D = L::D;
  const long long cell = (long long)blockIdx.x * kAuxThreads + threadIdx.x;
  if (cell >= g.n) return;
  int x, y, z;
  cell_coords(cell, g, x, y, z);
  const long long n = g.n;
  Macro m;
  m.rho = rho[cell];
  m.drho = m.rho - 1.0f;
  m.ux = u[cell];
  m.uy = u[n + cell];
  m.uz = D == 3 ? u[2 * n + cell] : 0.0f;
  m.jx = m.rho * m.ux;
  m.jy = m.rho * m.uy;
  m.jz = m.rho * m.uz;
  m.pxx = m.pxy = m.pxz = m.pyy = m.pyz = m.pzz = 0.0f;
  // nodes on a wall start at rest, f = f0(rho, 0)
  const bool wall = g.walls && unknown_mask<Q>(g, x, y, z) != 0;
  if (wall) {
    m.ux = m.uy = m.uz = 0.0f;
    m.jx = m.jy = m.jz = 0.0f;
  }
  if (mode == 1 && !wall) {
    // du[b][a] = d u_b / d x_a by periodic central differences
    float du[3][3] = {};
    const int p[3] = {x, y, z};
    const int dims[3] = {g.nx, g.ny, g.nz};
#pragma unroll
    for (int a = 0; a < D; ++a) {
      int pp[3] = {p[0], p[1], p[2]}, pm[3] = {p[0], p[1], p[2]};
      pp[a] = wrap_add(p[a], 1, dims[a]);
      pm[a] = wrap_add(p[a], -1, dims[a]);
      const long long cp = ((long long)pp[2] * g.ny + pp[1]) * g.nx + pp[0];
      const long long cm = ((long long)pm[2] * g.ny + pm[1]) * g.nx + pm[0];
#pragma unroll
      for (int b = 0; b < D; ++b) du[b][a] = 0.5f * (u[b * n + cp] - u[b * n + cm]);
    }
    const float k = -2.0f * kCs2 * m.rho * tau;
    m.pxx = k * du[0][0];
    m.pyy = k * du[1][1];
    m.pxy = k * 0.5f * (du[0][1] + du[1][0]);
    if (D == 3) {
      m.pzz = k * du[2][2];
      m.pxz = k * 0.5f * (du[0][2] + du[2][0]);
      m.pyz = k * 0.5f * (du[1][2] + du[2][1]);
    }
  }
  float df[Q];
  L::template synth<MODEL>(m, 1.0f, df);
#pragma unroll
  for (int i = 0; i < Q; ++i) Storage<S>::template store<Q>(f + i * n + cell, i, df[i]);
}

// ----------------------------------------------------------- populations --
template <int Q, int S>
__global__ void __launch_bounds__(kAuxThreads)
    get_populations_kernel(const typename Storage<S>::T *__restrict__ f, const Grid g,
                           const int parity, float *__restrict__ dst) {
  const long long cell = (long long)blockIdx.x * kAuxThreads + threadIdx.x;
  if (cell >= g.n) return;
  int x, y, z;
  cell_coords(cell, g, x, y, z);
  float df[Q];
  load_logical<Q, S>(f, g, parity, x, y, z, df);
#pragma unroll
  for (int i = 0; i < Q; ++i) dst[i * g.n + cell] = df[i];
}

template <int Q, int S>
__global__ void __launch_bounds__(kAuxThreads)
    set_populations_kernel(typename Storage<S>::T *__restrict__ f, const Grid g,
                           const float *__restrict__ src) {
  const long long cell = (long long)blockIdx.x * kAuxThreads + threadIdx.x;
  if (cell >= g.n) return;
#pragma unroll
  for (int i = 0; i < Q; ++i)
    Storage<S>::template store<Q>(f + i * g.n + cell, i, src[i * g.n + cell]);
}

// --------------------------------------------------------------- moments --
template <int Q, int S>
__global__ void __launch_bounds__(kAuxThreads)
    moments_kernel(const typename Storage<S>::T *__restrict__ f, const Grid g, const int parity,
                   float *__restrict__ rho, float *__restrict__ u, float *__restrict__ pi1) {
  constexpr int D = Lattice<Q>::D;
  const long long cell = (long long)blockIdx.x * kAuxThreads + threadIdx.x;
  if (cell >= g.n) return;
  int x, y, z;
  cell_coords(cell, g, x, y, z);
  float df[Q];
  load_logical<Q, S>(f, g, parity, x, y, z, df);
  // a node on a wall reports its closed state (rho of the fill, u = 0)
  const uint32_t unknown = g.walls ? unknown_mask<Q>(g, x, y, z) : 0u;
  if (unknown) wall_fill<Q>(unknown, df);
  Macro m = Lattice<Q>::moments(df);
  if (unknown) wall_macro(m);
  const long long n = g.n;
  if (rho) rho[cell] = m.rho;
  if (u) {
    u[cell] = m.ux;
    u[n + cell] = m.uy;
    if (D == 3) u[2 * n + cell] = m.uz;
  }
  if (pi1) {
    if (D == 2) {
      pi1[cell] = m.pxx;
      pi1[n + cell] = m.pxy;
      pi1[2 * n + cell] = m.pyy;
    } else {
      pi1[cell] = m.pxx;
      pi1[n + cell] = m.pxy;
      pi1[2 * n + cell] = m.pxz;
      pi1[3 * n + cell] = m.pyy;
      pi1[4 * n + cell] = m.pyz;
      pi1[5 * n + cell] = m.pzz;
    }
  }
}

// ------------------------------------------------------------ reductions --
// Block sum of NV doubles per thread: warp shuffles, then one value per warp
// in shared memory, then the first warp. The order is fixed, so results are
// reproducible run to run.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *out) {
  __shared__ double sm[kRedThreads / 32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sm[warp][k] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = lane < kRedThreads / 32 ? sm[lane][k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) out[k] = s;
    }
  }
}

// Mass, momentum and kinetic energy of the logical populations. Work items
// are chunks of kRedThreads cells of one row (y, z), a block taking items
// blockIdx.x, blockIdx.x + gridDim.x, ... and each thread one cell of the
// item. Logical population i of cell x is slot i at x (parity 0) or slot
// s = opp(i) at x + cx_s of row (y + cy_s, z + cz_s) (parity 1); the Q
// slot-row offsets are computed once per item. Per-cell values are formed in
// FP32 and summed over up to kDiagFlush cells in FP32, then accumulated in
// FP64 (FP64 arithmetic is slow on this GPU); the order is fixed, so results
// are reproducible run to run.
constexpr int kDiagFlush = 8;

template <int Q, int S, int PARITY>
__global__ void __launch_bounds__(kRedThreads)
    diag_partial_kernel(const typename Storage<S>::T *__restrict__ f, const Grid g,
                        double *__restrict__ partials) {
  constexpr int D = Lattice<Q>::D;
  __shared__ long long srow[Q];
  double acc[kRedValues] = {0.0, 0.0, 0.0, 0.0, 0.0};
  float part[kRedValues] = {0.f, 0.f, 0.f, 0.f, 0.f};
  int pending = 0;
  const int chunks = (g.nx + kRedThreads - 1) / kRedThreads;
  const long long items = (long long)g.ny * g.nz * chunks;
  for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const int r = (int)(it / chunks), x = (int)(it - (long long)r * chunks) * kRedThreads + threadIdx.x;
    __syncthreads();  // the previous item's offsets are no longer read
    if (threadIdx.x < Q) {
      const int sl = threadIdx.x;
      int y = r % g.ny, z = r / g.ny;
      if (PARITY) {
        y = wrap_add(y, vel_q<Q>(sl, 1), g.ny);
        z = D == 3 ? wrap_add(z, vel_q<Q>(sl, 2), g.nz) : 0;
      }
      srow[sl] = (long long)sl * g.n + ((long long)z * g.ny + y) * g.nx;
    }
    __syncthreads();
    if (x < g.nx) {
      const int xm = x == 0 ? g.nx - 1 : x - 1, xp = x + 1 == g.nx ? 0 : x + 1;
      float df[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const int sl = PARITY ? Q - 1 - i : i;
        const int cx = PARITY ? vel_q<Q>(sl, 0) : 0;
        const int xs = cx < 0 ? xm : (cx > 0 ? xp : x);
        df[i] = Storage<S>::template load<Q>(f + srow[sl] + xs, i);
      }
      const uint32_t unknown = g.walls ? unknown_mask<Q>(g, x, r % g.ny, r / g.ny) : 0u;
      if (unknown) wall_fill<Q>(unknown, df);
      Macro m = Lattice<Q>::moments(df);
      if (unknown) wall_macro(m);
      part[0] += m.drho;
      part[1] += m.jx;
      part[2] += m.jy;
      part[3] += m.jz;
      part[4] += 0.5f * (m.jx * m.ux + m.jy * m.uy + m.jz * m.uz);
      if (++pending == kDiagFlush) {
#pragma unroll
        for (int k = 0; k < kRedValues; ++k) {
          acc[k] += (double)part[k];
          part[k] = 0.f;
        }
        pending = 0;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kRedValues; ++k) acc[k] += (double)part[k];
  block_sum<kRedValues>(acc, partials + (long long)blockIdx.x * kRedValues);
}

// Sums nblocks rows of nv partials in a fixed order into out[nv].
__global__ void __launch_bounds__(kRedThreads)
    finalize_kernel(const double *__restrict__ partials, int nblocks, int nv,
                    double *__restrict__ out) {
  for (int k = 0; k < nv; ++k) {
    double v[1] = {0.0};
    for (int b = threadIdx.x; b < nblocks; b += kRedThreads) v[0] += partials[(long long)b * nv + k];
    __shared__ double res[1];
    block_sum<1>(v, res);
    __syncthreads();
    if (threadIdx.x == 0) out[k] = res[0];
    __syncthreads();
  }
}

// 0.5 |curl u|^2 per cell with periodic central differences.
template <int D>
__global__ void __launch_bounds__(kRedThreads)
    enstrophy_partial_kernel(const float *__restrict__ u, const Grid g,
                             double *__restrict__ partials) {
  double acc[1] = {0.0};
  const long long n = g.n;
  const long long stride = (long long)gridDim.x * kRedThreads;
  for (long long cell = (long long)blockIdx.x * kRedThreads + threadIdx.x; cell < n;
       cell += stride) {
    int x, y, z;
    cell_coords(cell, g, x, y, z);
    const int p[3] = {x, y, z}, dims[3] = {g.nx, g.ny, g.nz};
    // d u_comp / d x_axis: central differences (periodic across periodic
    // faces); second-order one-sided on the wall planes of a walled axis
    auto diff = [&](int comp, int axis) -> double {
      int q[3] = {p[0], p[1], p[2]};
      auto at = [&](int k) -> double {
        q[axis] = k;
        return (double)u[comp * n + ((long long)q[2] * g.ny + q[1]) * g.nx + q[0]];
      };
      const int a = p[axis], m = dims[axis];
      if ((g.walls >> axis) & 1) {
        if (a == 0) {
          const double u0 = at(0), u1 = at(1), u2 = at(2);
          return 0.5 * (-3.0 * u0 + 4.0 * u1 - u2);
        }
        if (a == m - 1) {
          const double u0 = at(m - 1), u1 = at(m - 2), u2 = at(m - 3);
          return 0.5 * (3.0 * u0 - 4.0 * u1 + u2);
        }
      }
      const double up = at(a + 1 == m ? 0 : a + 1);
      const double um = at(a == 0 ? m - 1 : a - 1);
      return 0.5 * (up - um);
    };
    double wgt = 1.0;
#pragma unroll
    for (int a = 0; a < D; ++a)
      if (((g.walls >> a) & 1) && (p[a] == 0 || p[a] == dims[a] - 1)) wgt *= 0.5;
    const double wz = diff(1, 0) - diff(0, 1);
    double wx = 0.0, wy = 0.0;
    if (D == 3) {
      wx = diff(2, 1) - diff(1, 2);
      wy = diff(0, 2) - diff(2, 0);
    }
    acc[0] += wgt * 0.5 * (wx * wx + wy * wy + wz * wz);
  }
  block_sum<1>(acc, partials + blockIdx.x);
}

// --------------------------------------------------------------- launchers --
static dim3 cells_grid(long long n) { return dim3((unsigned)((n + kAuxThreads - 1) / kAuxThreads)); }

static int red_blocks(long long n, int max_blocks) {
  long long b = (n + kRedThreads - 1) / kRedThreads;
  return (int)(b < max_blocks ? b : max_blocks);
}

// Calls fn(integral_constant<Q>, integral_constant<S>) for the runtime
// lattice size q and storage code.
template <class F>
static void dispatch_qs(int q, int storage, F &&fn) {
  using std::integral_constant;
  if (q == 9) {
    if (storage == 0) fn(integral_constant<int, 9>{}, integral_constant<int, 0>{});
    else if (storage == 1) fn(integral_constant<int, 9>{}, integral_constant<int, 1>{});
    else fn(integral_constant<int, 9>{}, integral_constant<int, 2>{});
  } else if (q == 19) {
    if (storage == 0) fn(integral_constant<int, 19>{}, integral_constant<int, 0>{});
    else if (storage == 1) fn(integral_constant<int, 19>{}, integral_constant<int, 1>{});
    else fn(integral_constant<int, 19>{}, integral_constant<int, 2>{});
  } else {
    if (storage == 0) fn(integral_constant<int, 27>{}, integral_constant<int, 0>{});
    else if (storage == 1) fn(integral_constant<int, 27>{}, integral_constant<int, 1>{});
    else fn(integral_constant<int, 27>{}, integral_constant<int, 2>{});
  }
}

cudaError_t launch_init(int q, int storage, int model, void *f, const Grid &g, const float *rho,
                        const float *u, float tau, int mode, cudaStream_t st) {
  dispatch_qs(q, storage, [&](auto qc, auto sc) {
    constexpr int Q_ = decltype(qc)::value;
    constexpr int S_ = decltype(sc)::value;
    using T = typename Storage<S_>::T;
    if (model != 1)  // RR and BGK contexts start from the full-basis f0 + f1
      init_kernel<Q_, S_, 0><<<cells_grid(g.n), kAuxThreads, 0, st>>>(static_cast<T *>(f), g,
                                                                        rho, u, tau, mode);
    else
      init_kernel<Q_, S_, 1><<<cells_grid(g.n), kAuxThreads, 0, st>>>(static_cast<T *>(f), g,
                                                                        rho, u, tau, mode);
  });
  return cudaGetLastError();
}

cudaError_t launch_get_populations(int q, int storage, const void *f, const Grid &g, int parity,
                                   float *dst, cudaStream_t st) {
  dispatch_qs(q, storage, [&](auto qc, auto sc) {
    constexpr int Q_ = decltype(qc)::value;
    constexpr int S_ = decltype(sc)::value;
    using T = typename Storage<S_>::T;
    get_populations_kernel<Q_, S_><<<cells_grid(g.n), kAuxThreads, 0, st>>>(
        static_cast<const T *>(f), g, parity, dst);
  });
  return cudaGetLastError();
}

cudaError_t launch_set_populations(int q, int storage, void *f, const Grid &g, const float *src,
                                   cudaStream_t st) {
  dispatch_qs(q, storage, [&](auto qc, auto sc) {
    constexpr int Q_ = decltype(qc)::value;
    constexpr int S_ = decltype(sc)::value;
    using T = typename Storage<S_>::T;
    set_populations_kernel<Q_, S_><<<cells_grid(g.n), kAuxThreads, 0, st>>>(static_cast<T *>(f),
                                                                            g, src);
  });
  return cudaGetLastError();
}

cudaError_t launch_moments(int q, int storage, const void *f, const Grid &g, int parity,
                           float *rho, float *u, float *pi1, cudaStream_t st) {
  dispatch_qs(q, storage, [&](auto qc, auto sc) {
    constexpr int Q_ = decltype(qc)::value;
    constexpr int S_ = decltype(sc)::value;
    using T = typename Storage<S_>::T;
    moments_kernel<Q_, S_><<<cells_grid(g.n), kAuxThreads, 0, st>>>(static_cast<const T *>(f), g,
                                                                     parity, rho, u, pi1);
  });
  return cudaGetLastError();
}

cudaError_t launch_diagnostics(int q, int storage, const void *f, const Grid &g, int parity,
                               int max_blocks, double *partials, double *out, cudaStream_t st) {
  const int nb = red_blocks(g.n, max_blocks);
  dispatch_qs(q, storage, [&](auto qc, auto sc) {
    constexpr int Q_ = decltype(qc)::value;
    constexpr int S_ = decltype(sc)::value;
    using T = typename Storage<S_>::T;
    if (parity)
      diag_partial_kernel<Q_, S_, 1><<<nb, kRedThreads, 0, st>>>(static_cast<const T *>(f), g,
                                                                 partials);
    else
      diag_partial_kernel<Q_, S_, 0><<<nb, kRedThreads, 0, st>>>(static_cast<const T *>(f), g,
                                                                 partials);
  });
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  finalize_kernel<<<1, kRedThreads, 0, st>>>(partials, nb, kRedValues, out);
  return cudaGetLastError();
}

cudaError_t launch_diagnostics_blocks(int q, int storage, const void *f, const Grid &g,
                                      int parity, int nblocks, double *partials, double *out,
                                      cudaStream_t st) {
  dispatch_qs(q, storage, [&](auto qc, auto sc) {
    constexpr int Q_ = decltype(qc)::value;
    constexpr int S_ = decltype(sc)::value;
    using T = typename Storage<S_>::T;
    if (parity)
      diag_partial_kernel<Q_, S_, 1><<<nblocks, kRedThreads, 0, st>>>(static_cast<const T *>(f),
                                                                      g, partials);
    else
      diag_partial_kernel<Q_, S_, 0><<<nblocks, kRedThreads, 0, st>>>(static_cast<const T *>(f),
                                                                      g, partials);
  });
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  finalize_kernel<<<1, kRedThreads, 0, st>>>(partials, nblocks, kRedValues, out);
  return cudaGetLastError();
}

cudaError_t launch_enstrophy(int d, const float *u, const Grid &g, int max_blocks,
                             double *partials, double *out, cudaStream_t st) {
  const int nb = red_blocks(g.n, max_blocks);
  if (d == 2)
    enstrophy_partial_kernel<2><<<nb, kRedThreads, 0, st>>>(u, g, partials);
  else
    enstrophy_partial_kernel<3><<<nb, kRedThreads, 0, st>>>(u, g, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  finalize_kernel<<<1, kRedThreads, 0, st>>>(partials, nb, 1, out);
  return cudaGetLastError();
}

}  // namespace lbrr
