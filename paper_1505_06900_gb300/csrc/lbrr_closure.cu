// Learned closure on the RR step (an extension; the paper has no learned
// component): moment field, standardised features and targets for training,
// 2x2x2 coarsening of a fine run, and the update of a coarse D3Q27 FP32 store
// in which the network's prediction of the order 3..6 off-equilibrium
// coefficients is added to the recursion's before the (1 - 1/tau)
// relaxation.
//
// Feature of a cell: the moments (rho - 1, u, Pi1) of the cell and its 26
// periodic neighbours, standardised per moment kind, neighbour index
// (dx+1) + 3(dy+1) + 9(dz+1), feature 10 * neighbour + moment, zero padded
// to 288. Target: the order 3..6 Hermite coefficients of (f - f_RR), f_RR the
// RR reconstruction from the cell's own moments, divided by out_scale, in the
// order xxy, xxz, xyy, xzz, yzz, yyz, xyz, xxyy, xxzz, yyzz, xyzz, xyyz, xxyz,
// xxyzz, xxyyz, xyyzz, xxyyzz, zero padded to 32.
#include "lbrr_launch.h"
#include "lbrr_mlp.h"
#include "lbrr_act.cuh"

namespace lbrr {

namespace {

constexpr int kAux = 128;

// --------------------------------------------------------------- moments --
__global__ void __launch_bounds__(kAux)
    moment_field_kernel(const float *__restrict__ f, const Grid g, const int parity,
                        float *__restrict__ mom) {
  const long long cell = (long long)blockIdx.x * kAux + threadIdx.x;
  if (cell >= g.n) return;
  int x, y, z;
  cell_coords(cell, g, x, y, z);
  float df[27];
  load_logical<27, 0>(f, g, parity, x, y, z, df);
  const Macro m = Lattice<27>::moments(df);
  const long long n = g.n;
  const float v[kMlpMoments] = {m.drho, m.ux, m.uy, m.uz, m.pxx, m.pxy, m.pxz, m.pyy, m.pyz, m.pzz};
#pragma unroll
  for (int k = 0; k < kMlpMoments; ++k) mom[k * n + cell] = v[k];
}

// -------------------------------------------------------------- features --
__device__ __forceinline__ long long nb_cell(const Grid &g, int x, int y, int z, int nb) {
  const int dx = nb % 3 - 1, dy = (nb / 3) % 3 - 1, dz = nb / 9 - 1;
  return ((long long)wrap_add(z, dz, g.nz) * g.ny + wrap_add(y, dy, g.ny)) * g.nx +
         wrap_add(x, dx, g.nx);
}

__global__ void __launch_bounds__(kAux)
    features_kernel(MlpDevice p, const float *__restrict__ mom, const Grid g,
                    __nv_bfloat16 *__restrict__ X) {
  const long long cell = (long long)blockIdx.x * kAux + threadIdx.x;
  if (cell >= g.n) return;
  int x, y, z;
  cell_coords(cell, g, x, y, z);
  const long long n = g.n;
  uint32_t *row = reinterpret_cast<uint32_t *>(X + cell * kMlpIn);
  for (int nb = 0; nb < 27; ++nb) {
    const long long c = nb_cell(g, x, y, z, nb);
#pragma unroll
    for (int k = 0; k < kMlpMoments; k += 2) {
      const float v0 = (__ldg(mom + k * n + c) - p.in_mean[k]) * p.in_inv_std[k];
      const float v1 = (__ldg(mom + (k + 1) * n + c) - p.in_mean[k + 1]) * p.in_inv_std[k + 1];
      row[(kMlpMoments * nb + k) / 2] = pack_bf16(v0, v1);
    }
  }
  for (int k = kMlpInUsed; k < kMlpIn; k += 2) row[k / 2] = 0u;
}

// --------------------------------------------------------------- targets --
// 1-D Hermite analysis of a line d(-1), d(0), d(+1): sums of H0 = 1,
// H1 = xi, H2 = xi^2 - 1/3 times d.
__device__ __forceinline__ void ana1(float dm, float dz, float dp, float &e0, float &e1,
                                     float &e2) {
  e0 = dm + dz + dp;
  e1 = dp - dm;
  e2 = fmaf(2.0f / 3.0f, dm + dp, -dz / 3.0f);
}

// Hermite coefficients A[a][b][c] = sum_i H_a(xi_x) H_b(xi_y) H_c(xi_z) d_i of
// a D3Q27 population vector (separable: x lines, then y, then z).
__device__ __forceinline__ void hermite_analysis(const float (&d)[27], float (&A)[3][3][3]) {
  float ax[3][9];  // [a][line (iy, iz)]
#pragma unroll
  for (int l = 0; l < 9; ++l) ana1(d[3 * l], d[3 * l + 1], d[3 * l + 2], ax[0][l], ax[1][l], ax[2][l]);
  float axy[3][3][3];  // [a][b][iz]
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int iz = 0; iz < 3; ++iz)
      ana1(ax[a][3 * iz], ax[a][3 * iz + 1], ax[a][3 * iz + 2], axy[a][0][iz], axy[a][1][iz],
           axy[a][2][iz]);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      ana1(axy[a][b][0], axy[a][b][1], axy[a][b][2], A[a][b][0], A[a][b][1], A[a][b][2]);
}

// Row `cell` of a target matrix: the order 3..6 coefficients of A divided by
// div * out_scale, zero padded.
__device__ __forceinline__ void write_targets(const MlpDevice &p, const float (&A)[3][3][3],
                                              float div, float *__restrict__ row) {
#pragma unroll
  for (int k = 0; k < kMlpOutUsed; ++k)
    row[k] = A[hi_pow(k, 0)][hi_pow(k, 1)][hi_pow(k, 2)] / (div * p.out_scale[k]);
  for (int k = kMlpOutUsed; k < kMlpOut; ++k) row[k] = 0.f;
}

__global__ void __launch_bounds__(kAux)
    targets_kernel(MlpDevice p, const float *__restrict__ f, const Grid g, const int parity,
                   float *__restrict__ T) {
  const long long cell = (long long)blockIdx.x * kAux + threadIdx.x;
  if (cell >= g.n) return;
  int x, y, z;
  cell_coords(cell, g, x, y, z);
  float df[27], rr[27];
  load_logical<27, 0>(f, g, parity, x, y, z, df);
  const Macro m = Lattice<27>::moments(df);
  Lattice<27>::synth<0>(m, 1.0f, rr);  // f_RR - w (tau -> infinity)
#pragma unroll
  for (int i = 0; i < 27; ++i) rr[i] = df[i] - rr[i];
  float A[3][3][3];
  hermite_analysis(rr, A);
  write_targets(p, A, 1.0f, T + cell * kMlpOut);
}

// Step-matching targets of coarse cell x: P_i(x) = post_i(x + xi_i) (logical
// populations; in the AA store, parity 0: slot i of x + xi_i, parity 1: slot
// opp(i) of x itself), R = the RR post-collision of pre's cell x; the order
// 3..6 coefficients of (P - R) / om1. Shifted values throughout: the weights
// cancel in the difference.
__global__ void __launch_bounds__(kAux)
    step_targets_kernel(MlpDevice p, const float *__restrict__ fpre, const int ppre,
                        const float *__restrict__ fpost, const int ppost, const Grid g,
                        const float om1, float *__restrict__ T) {
  const long long cell = (long long)blockIdx.x * kAux + threadIdx.x;
  if (cell >= g.n) return;
  int x, y, z;
  cell_coords(cell, g, x, y, z);
  float df[27], r[27];
  load_logical<27, 0>(fpre, g, ppre, x, y, z, df);
  const Macro m = Lattice<27>::moments(df);
  Lattice<27>::synth<0>(m, om1, r);
  const long long n = g.n;
#pragma unroll
  for (int i = 0; i < 27; ++i) {
    float pi;
    if (ppost == 0) {
      const long long dst = ((long long)wrap_add(z, vel(i, 2), g.nz) * g.ny +
                             wrap_add(y, vel(i, 1), g.ny)) * g.nx + wrap_add(x, vel(i, 0), g.nx);
      pi = __ldg(fpost + i * n + dst);
    } else {
      pi = __ldg(fpost + (26 - i) * n + cell);
    }
    r[i] = pi - r[i];
  }
  float A[3][3][3];
  hermite_analysis(r, A);
  write_targets(p, A, om1, T + cell * kMlpOut);
}

// -------------------------------------------------------------- coarsen --
// RESCALE: the off-equilibrium part of the average is scaled,
// f0(rho, u) + scale (fbar - f0(rho, u)) with rho, u the moments of fbar.
template <int SF, int SC, bool RESCALE = false>
__global__ void __launch_bounds__(kAux)
    coarsen_kernel(const typename Storage<SF>::T *__restrict__ ff, const Grid gf, const int parity,
                   typename Storage<SC>::T *__restrict__ fc, const Grid gc, const float scale) {
  const long long cell = (long long)blockIdx.x * kAux + threadIdx.x;
  if (cell >= gc.n) return;
  int x, y, z;
  cell_coords(cell, gc, x, y, z);
  float acc[27] = {};
#pragma unroll 1
  for (int s = 0; s < 8; ++s) {
    float df[27];
    load_logical<27, SF>(ff, gf, parity, 2 * x + (s & 1), 2 * y + ((s >> 1) & 1),
                         2 * z + (s >> 2), df);
#pragma unroll
    for (int i = 0; i < 27; ++i) acc[i] += df[i];
  }
#pragma unroll
  for (int i = 0; i < 27; ++i) acc[i] *= 0.125f;
  if (RESCALE) {
    const Macro m = Lattice<27>::moments(acc);
    float eq[27];
    Lattice<27>::synth<0>(m, 0.0f, eq);  // f0 - w
#pragma unroll
    for (int i = 0; i < 27; ++i) acc[i] = fmaf(scale, acc[i] - eq[i], eq[i]);
  }
#pragma unroll
  for (int i = 0; i < 27; ++i) Storage<SC>::template store<27>(fc + i * gc.n + cell, i, acc[i]);
}

// ---------------------------------------------------------- closure step --
// One thread per cell (blocks along x, AA parity as in lbrr_step.cu): RR
// coefficients plus (1 - 1/tau) times the network's correction, RR alone for
// a cell whose standardised prediction exceeds the bound or whose corrected
// populations are not all positive (counted).
constexpr int kDT = 128;

template <int PARITY>
__global__ void __launch_bounds__(kDT)
    rr_step_delta_kernel(MlpDevice p, float *__restrict__ f, const Grid g, const float om1,
                         const float *__restrict__ ystd, unsigned long long *fallbacks,
                         const float bound, const float dead_zone) {
  const int x = blockIdx.x * kDT + threadIdx.x;
  if (x >= g.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const long long cell = ((long long)z * g.ny + y) * g.nx + x;
  float yk[kMlpOutUsed];
#pragma unroll
  for (int k = 0; k < kMlpOutUsed; ++k) yk[k] = __ldg(ystd + k * g.n + cell);
  closure_update_cell<PARITY>(p, f, g, om1, x, y, z, yk, fallbacks, bound, dead_zone);
}

}  // namespace

cudaError_t launch_moment_field(int storage, const void *f, const Grid &g, int parity, float *mom,
                                cudaStream_t st) {
  if (storage != 0) return cudaErrorInvalidValue;
  moment_field_kernel<<<(unsigned)((g.n + kAux - 1) / kAux), kAux, 0, st>>>(
      static_cast<const float *>(f), g, parity, mom);
  return cudaGetLastError();
}

cudaError_t launch_features(const MlpDevice &p, const float *mom, const Grid &g, void *X,
                            cudaStream_t st) {
  features_kernel<<<(unsigned)((g.n + kAux - 1) / kAux), kAux, 0, st>>>(
      p, mom, g, static_cast<__nv_bfloat16 *>(X));
  return cudaGetLastError();
}

cudaError_t launch_targets(const MlpDevice &p, int storage, const void *f, const Grid &g,
                           int parity, float *T, cudaStream_t st) {
  if (storage != 0) return cudaErrorInvalidValue;
  targets_kernel<<<(unsigned)((g.n + kAux - 1) / kAux), kAux, 0, st>>>(
      p, static_cast<const float *>(f), g, parity, T);
  return cudaGetLastError();
}

cudaError_t launch_coarsen(int storage_f, const void *ff, const Grid &gf, int parity_f,
                           int storage_c, void *fc, const Grid &gc, cudaStream_t st,
                           float neq_scale) {
  const unsigned nb = (unsigned)((gc.n + kAux - 1) / kAux);
  if (storage_f != 0 || storage_c != 0) return cudaErrorInvalidValue;
  if (neq_scale == 1.0f)
    coarsen_kernel<0, 0><<<nb, kAux, 0, st>>>(static_cast<const float *>(ff), gf, parity_f,
                                              static_cast<float *>(fc), gc, 1.0f);
  else
    coarsen_kernel<0, 0, true><<<nb, kAux, 0, st>>>(static_cast<const float *>(ff), gf, parity_f,
                                                    static_cast<float *>(fc), gc, neq_scale);
  return cudaGetLastError();
}

cudaError_t launch_step_targets(const MlpDevice &p, const float *fpre, int ppre,
                                const float *fpost, int ppost, const Grid &g, float om1, float *T,
                                cudaStream_t st) {
  step_targets_kernel<<<(unsigned)((g.n + kAux - 1) / kAux), kAux, 0, st>>>(p, fpre, ppre, fpost,
                                                                           ppost, g, om1, T);
  return cudaGetLastError();
}

cudaError_t launch_step_delta(const MlpDevice &p, float *f, const Grid &g, float om1, int parity,
                              const float *ystd, unsigned long long *fallbacks, float bound,
                              float dead_zone, cudaStream_t st) {
  const dim3 grid((g.nx + kDT - 1) / kDT, g.ny, g.nz);
  if (parity == 0)
    rr_step_delta_kernel<0><<<grid, kDT, 0, st>>>(p, f, g, om1, ystd, fallbacks, bound,
                                                 dead_zone);
  else
    rr_step_delta_kernel<1><<<grid, kDT, 0, st>>>(p, f, g, om1, ystd, fallbacks, bound,
                                                 dead_zone);
  return cudaGetLastError();
}

}  // namespace lbrr
