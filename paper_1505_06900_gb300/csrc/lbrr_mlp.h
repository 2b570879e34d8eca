// Internal declarations of the learned closure (network kernels, feature and
// target extraction, coarsening, the closure step). Not part of the C ABI.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "lbrr_device.cuh"

namespace lbrr {

constexpr int kMlpIn = 288;      // 27 cells x 10 moments = 270 features, zero padded
constexpr int kMlpInUsed = 270;
constexpr int kMlpHidden = 64;
constexpr int kMlpOut = 32;      // 17 coefficients of orders 3..6, zero padded
constexpr int kMlpOutUsed = 17;
constexpr int kMlpMoments = 10;  // rho - 1, ux, uy, uz, Pi xx, xy, xz, yy, yz, zz

// packed parameter layout: W1 [64][288], b1, W2 [64][64], b2, W3 [32][64], b3
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kMlpHidden * kMlpIn;
constexpr int kOffW2 = kOffB1 + kMlpHidden;
constexpr int kOffB2 = kOffW2 + kMlpHidden * kMlpHidden;
constexpr int kOffW3 = kOffB2 + kMlpHidden;
constexpr int kOffB3 = kOffW3 + kMlpOut * kMlpHidden;
constexpr int kMlpParams = kOffB3 + kMlpOut;  // 24736

// Device view of one network: FP32 master parameters and Adam moments, BF16
// copies of the weights in K-major layout (row = output unit) for the forward
// products and transposed copies of W2 and W3 for the backward products, and
// the feature / target standardisation.
struct MlpDevice {
  float *params, *adam_m, *adam_v;
  __nv_bfloat16 *w1, *w2, *w3, *w2t, *w3t;
  const float *b1, *b2, *b3;      // point into params
  const float *in_mean;           // [10]
  const float *in_inv_std;        // [10]
  const float *out_scale;         // [17]
};

__device__ void mlp_refresh_one(MlpDevice p, int k, float w);

// (a, b, c) powers of x^a y^b z^c of the 17 high-order coefficients, in the
// order of the network's outputs (xxy, xxz, xyy, xzz, yzz, yyz, xyz, xxyy,
// xxzz, yyzz, xyzz, xyyz, xxyz, xxyzz, xxyyz, xyyzz, xxyyzz)
__host__ __device__ constexpr int hi_pow(int k, int axis) {
  // packed as a + 3 b + 9 c
  constexpr int code[17] = {2 + 3 * 1,     2 + 9 * 1,     1 + 3 * 2,     1 + 9 * 2,
                            3 * 1 + 9 * 2, 3 * 2 + 9 * 1, 1 + 3 + 9,     2 + 3 * 2,
                            2 + 9 * 2,     3 * 2 + 9 * 2, 1 + 3 + 9 * 2, 1 + 3 * 2 + 9,
                            2 + 3 + 9,     2 + 3 + 9 * 2, 2 + 3 * 2 + 9, 1 + 3 * 2 + 9 * 2,
                            2 + 3 * 2 + 9 * 2};
  return axis == 0 ? code[k] % 3 : (axis == 1 ? (code[k] / 3) % 3 : code[k] / 9);
}

// Element offset of the location from which the update of cell (x, y, z) of
// an FP32 D3Q27 AA store (parity as in lbrr_step.cu) reads population i; the
// update writes population i to the location it_writes(i) below, and the two
// sets are the same 27 locations. IDX is the type of the element offsets:
// int needs 27 N < 2^31 (fewer registers).
template <int PARITY, typename IDX = long long>
__device__ __forceinline__ IDX closure_read_offset(const Grid &g, int x, int y, int z, int i) {
  const IDX n = (IDX)g.n;
  if (PARITY == 0) return (IDX)i * n + ((IDX)z * g.ny + y) * g.nx + x;
  const int xa = wrap_add(x, -vel(i, 0), g.nx), ya = wrap_add(y, -vel(i, 1), g.ny),
            za = wrap_add(z, -vel(i, 2), g.nz);
  return (IDX)(26 - i) * n + ((IDX)za * g.ny + ya) * g.nx + xa;
}

// The closure update of cell (x, y, z) of an FP32 D3Q27 AA store from its 27
// logical populations df (read at closure_read_offset): the RR coefficients
// plus (1 - 1/tau) times the network's correction, y'[k] out_scale[k] added
// to coefficient k of orders 3..6, with y' = sign(y) max(|y| - dead_zone, 0)
// the standardised prediction y = ystd[k] shrunk by the dead zone; plain RR
// for the cell (counted in *fallbacks) when a standardised prediction exceeds
// the bound (or is not a number) or a corrected population is not positive.
// Each cell writes exactly the locations it reads. out_scale: the 17
// scales (device or shared memory).
template <int PARITY, typename IDX = long long>
__device__ __forceinline__ void closure_update_cell_df(const float *out_scale,
                                                       float *__restrict__ f, const Grid &g,
                                                       const float om1, int x, int y, int z,
                                                       const float (&df)[27],
                                                       const float (&ystd)[kMlpOutUsed],
                                                       unsigned long long *fallbacks,
                                                       const float bound, const float dead_zone) {
  const Macro m = Lattice<27>::moments(df);
  bool use = true;
  float cc[3][3][3];
  coeffs_rr_d3q27(m, om1, cc);
#pragma unroll
  for (int k = 0; k < kMlpOutUsed; ++k) {
    const float yk = ystd[k];
    use = use && (fabsf(yk) <= bound);  // also false for NaN
    const float yd = copysignf(fmaxf(fabsf(yk) - dead_zone, 0.0f), yk);
    cc[hi_pow(k, 0)][hi_pow(k, 1)][hi_pow(k, 2)] += om1 * (yd * out_scale[k]);
  }
  float out[27];
  if (use) {
    synth_tensor_d3q27<false>(cc, out);
#pragma unroll
    // f_i = out[i] + w_i > 0, compared as out[i] > -w_i: the same test, since
    // near the boundary the sum of the two is exact (Sterbenz)
    for (int i = 0; i < 27; ++i) use = use && (out[i] > -weight<3>(i));
  }
  if (!use) {  // plain RR: the coefficients again from the moments (rare)
    coeffs_rr_d3q27(m, om1, cc);
    synth_tensor_d3q27<false>(cc, out);
    if (fallbacks) atomicAdd(fallbacks, 1ull);
  }
  const IDX n = (IDX)g.n;
  const int xs3[3] = {wrap_add(x, -1, g.nx), x, wrap_add(x, 1, g.nx)};
  const int ys3[3] = {wrap_add(y, -1, g.ny), y, wrap_add(y, 1, g.ny)};
  const int zs3[3] = {wrap_add(z, -1, g.nz), z, wrap_add(z, 1, g.nz)};
  auto cell_at = [&](int b, int c, int a) -> IDX {
    return ((IDX)zs3[c] * g.ny + ys3[b]) * g.nx + xs3[a];
  };
  const IDX cell = cell_at(1, 1, 1);
#pragma unroll
  for (int i = 0; i < 27; ++i) {
    if (PARITY == 0)
      f[(26 - i) * n + cell] = out[i];
    else
      f[i * n + cell_at(1 + vel(i, 1), 1 + vel(i, 2), 1 + vel(i, 0))] = out[i];
  }
}

// The same, reading the populations itself.
template <int PARITY, typename IDX = long long>
__device__ __forceinline__ void closure_update_cell(const MlpDevice &p, float *__restrict__ f,
                                                    const Grid &g, const float om1, int x, int y,
                                                    int z, const float (&ystd)[kMlpOutUsed],
                                                    unsigned long long *fallbacks,
                                                    const float bound, const float dead_zone) {
  float df[27];
#pragma unroll
  for (int i = 0; i < 27; ++i) df[i] = f[closure_read_offset<PARITY, IDX>(g, x, y, z, i)];
  closure_update_cell_df<PARITY, IDX>(p.out_scale, f, g, om1, x, y, z, df, ystd, fallbacks,
                                      bound, dead_zone);
}

constexpr int kMlpTrainRows = 128;  // batch rows per tile of the training kernel

// Columns of one trace row of the training kernel (FP32, as computed, before
// any BF16 rounding): layer-1 and layer-2 activations, outputs, the loss
// gradient dy = 2 (y - t) / (17 M) on the used outputs, and the back-propagated
// dh2 = (W3^T dy) (1 - h2^2), dh1 = (W2^T dh2) (1 - h1^2).
constexpr int kTraceH1 = 0, kTraceH2 = 64, kTraceY = 128, kTraceDy = 160, kTraceDh2 = 192,
              kTraceDh1 = 256, kMlpTrace = 320;

// Forward + backward of a batch on the tcgen05 tensor cores (lbrr_mlp_train.cu):
// writes the block partial gradients gpart [b][kMlpParams] and loss sums
// lpart[b] of the min(nblocks, tiles of kMlpTrainRows rows) blocks; with
// trace also the trace rows [M][kMlpTrace]. *status becomes 1 if a
// tensor-core wait timed out (the partials are then incomplete).
cudaError_t launch_mlp_train(const MlpDevice &p, const void *X, const float *T, long long M,
                             float *gpart, float *lpart, int *status, int nblocks,
                             cudaStream_t st, float *trace = nullptr);
// Gradient = sum of the partials; optional Adam step (bias corrections bc1,
// bc2); loss = sum of the block losses (double, device) when loss_out != null.
// Nothing is updated while *status (the training kernel's timeout flag) is set.
cudaError_t launch_mlp_reduce(const MlpDevice &p, const float *gpart, int nparts, float *grad_out,
                              int adam, float lr, float bc1, float bc2, const float *lpart,
                              double *loss_out, const int *status, cudaStream_t st);
cudaError_t launch_mlp_refresh(const MlpDevice &p, cudaStream_t st);

// Moment field [10][N] of the logical populations (FP32 store only).
cudaError_t launch_moment_field(int storage, const void *f, const Grid &g, int parity, float *mom,
                                cudaStream_t st);
// Standardised features X [N][288] (BF16) from a moment field.
cudaError_t launch_features(const MlpDevice &p, const float *mom, const Grid &g, void *X,
                            cudaStream_t st);
// Standardised targets T [N][32] of the current populations.
cudaError_t launch_targets(const MlpDevice &p, int storage, const void *f, const Grid &g,
                           int parity, float *T, cudaStream_t st);
// 2x2x2 box average of a fine store into a coarse store (natural order),
// the off-equilibrium part scaled by neq_scale (1: the plain average).
cudaError_t launch_coarsen(int storage_f, const void *ff, const Grid &gf, int parity_f,
                           int storage_c, void *fc, const Grid &gc, cudaStream_t st,
                           float neq_scale = 1.0f);
// Standardised step-matching targets T [N][32] of the coarse state fpre
// against fpost (FP32 stores with their AA parities), om1 = 1 - 1/tau.
cudaError_t launch_step_targets(const MlpDevice &p, const float *fpre, int ppre,
                                const float *fpost, int ppost, const Grid &g, float om1, float *T,
                                cudaStream_t st);
// Network forward on the tcgen05 tensor cores (lbrr_mlp_tc.cu). With mom:
// rows are the cells of grid *g, features from the moment field, outputs the
// 17 standardised predictions Y [17][N]. Without: rows X [M][288] BF16, Y
// [M][32]. *status becomes 1 if a tensor-core wait timed out.
// With H (rows X only): also the FP32 activations of layers 1 and 2 of
// every row, H [M][128], as computed before their BF16 rounding.
cudaError_t launch_mlp_tc(const MlpDevice &p, const void *X, const float *mom, const Grid *g,
                          long long M, float *Y, int *status, int nblocks, cudaStream_t st,
                          float *H = nullptr);
// The TMA-fed, pipelined forward pass (lbrr_mlp_conv.cu) for grids whose
// rows are whole 128-cell tiles: the feature source xs (standardised moments,
// BF16, one-cell periodic halo, in the two 8-channel halves that kernel
// reads: feature_source_bytes(g) bytes), its tensor map, and the network on
// it. launch_export_features writes the feature source channels-last,
// [(nx + 2)(ny + 2)(nz + 2)][16] BF16 (channels 10..15 zero).
bool mlp_conv_supported(const Grid &g);
size_t feature_source_bytes(const Grid &g);
cudaError_t make_feature_map(void *xs, const Grid &g, CUtensorMap *map);
cudaError_t launch_feature_source(const MlpDevice &p, const float *f, const Grid &g, int parity,
                                  void *xs, cudaStream_t st);
cudaError_t launch_export_features(const void *xs, const Grid &g, void *out, cudaStream_t st);
// The network fused with the closure update: the thread that owns a
// tile row takes its cell's 17 predictions from the layer-3 accumulator and
// updates the cell in place (closure_update_cell), so no prediction goes
// through device memory. On a timeout (*status = 1) part of the cells have
// not been updated.
// With trace (inspection only): also trace [N][kConvTrace] per cell: the
// FP32 activations of layers 1 and 2 and the 17 standardised predictions.
constexpr int kConvTrace = 2 * kMlpHidden + kMlpOutUsed;  // 145
cudaError_t launch_mlp_conv_step(const MlpDevice &p, const CUtensorMap &map, const Grid &g,
                                 float *f, float om1, int parity, unsigned long long *fallbacks,
                                 float bound, float dead_zone, int *status, int nblocks,
                                 cudaStream_t st, float *trace = nullptr);
// One update of an FP32 D3Q27 store with the learned correction: ystd [17][N]
// holds the network's standardised predictions for the current populations.
cudaError_t launch_step_delta(const MlpDevice &p, float *f, const Grid &g, float om1, int parity,
                              const float *ystd, unsigned long long *fallbacks, float bound,
                              float dead_zone, cudaStream_t st);

}  // namespace lbrr
