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

size_t mlp_train_smem();

// Forward (T == nullptr: writes Y [M][32]) or forward + backward (writes the
// block partial gradients gpart [nblocks][kMlpParams] and losses lpart).
cudaError_t launch_mlp(const MlpDevice &p, const void *X, const float *T, long long M, float *Y,
                       float *gpart, float *lpart, int nblocks, cudaStream_t st);
// Gradient = sum of the partials; optional Adam step (bias corrections bc1,
// bc2); loss = sum of the block losses (double, device) when loss_out != null.
cudaError_t launch_mlp_reduce(const MlpDevice &p, const float *gpart, int nparts, float *grad_out,
                              int adam, float lr, float bc1, float bc2, const float *lpart,
                              double *loss_out, cudaStream_t st);
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
// 2x2x2 box average of a fine store into a coarse store (natural order).
cudaError_t launch_coarsen(int storage_f, const void *ff, const Grid &gf, int parity_f,
                           int storage_c, void *fc, const Grid &gc, cudaStream_t st);
// Network forward on the tcgen05 tensor cores (lbrr_mlp_tc.cu). With mom:
// rows are the cells of grid *g, features from the moment field, outputs the
// 17 standardised predictions Y [17][N]. Without: rows X [M][288] BF16, Y
// [M][32]. *status becomes 1 if a tensor-core wait timed out.
cudaError_t launch_mlp_tc(const MlpDevice &p, const void *X, const float *mom, const Grid *g,
                          long long M, float *Y, int *status, int nblocks, cudaStream_t st);
// The TMA-fed, pipelined forward pass (lbrr_mlp_conv.cu) for grids whose
// rows are whole 128-cell tiles: the feature source xs (standardised moments,
// BF16, 16 channels, one-cell periodic halo: feature_source_bytes(g) bytes),
// its tensor map, and the network on it writing Y [17][N].
bool mlp_conv_supported(const Grid &g);
size_t feature_source_bytes(const Grid &g);
cudaError_t make_feature_map(void *xs, const Grid &g, CUtensorMap *map);
cudaError_t launch_feature_source(const MlpDevice &p, const float *f, const Grid &g, int parity,
                                  void *xs, cudaStream_t st);
cudaError_t launch_mlp_conv(const MlpDevice &p, const CUtensorMap &map, const Grid &g, float *Y,
                            int *status, int nblocks, cudaStream_t st);
// One update of an FP32 D3Q27 store with the learned correction: ystd [17][N]
// holds the network's standardised predictions for the current populations.
cudaError_t launch_step_delta(const MlpDevice &p, float *f, const Grid &g, float om1, int parity,
                              const float *ystd, unsigned long long *fallbacks, float bound,
                              cudaStream_t st);

}  // namespace lbrr
