// Host-side launchers of the CUDA kernels (internal to liblbrr.so).
#pragma once

#include <cuda_runtime.h>

#include "lbrr_device.cuh"

namespace lbrr {

// Partial-sum blocks of the deterministic reductions per SM of the device
// (a context sizes its scratch as kRedBlocksPerSm x its device's SM count).
constexpr int kRedBlocksPerSm = 8;
constexpr int kRedThreads = 256;
constexpr int kRedValues = 5;      // partial sums per block (mass, momentum x3, energy)

// One collide-and-stream update of the AA store `f` (element type given by
// `storage`): parity 0 reads and writes the cell's own slots (writing the
// post-collision population i into slot opp(i)); parity 1 reads slot opp(i)
// of x - xi_i and writes slot i of x + xi_i. *status becomes 1 if a bounded
// wait of the 16-bit row kernel expired (the update is then incomplete).
cudaError_t launch_step(int q, int storage, int model, void *f, const Grid &g, float om1,
                        int parity, int *status, cudaStream_t st);

// The one-thread-per-cell kernel of launch_step (lbrr_step.cu), for any grid
// without walls and any storage.
cudaError_t launch_step_cell(int q, int storage, int model, void *f, const Grid &g, float om1,
                             int parity, cudaStream_t st);

// The update of a grid with no-slip walls (g.walls != 0; lbrr_walls.cu),
// any storage; launch_step dispatches to it.
cudaError_t launch_step_walls(int q, int storage, int model, void *f, const Grid &g, float om1,
                              int parity, cudaStream_t st);

// The persistent row kernel for 16-bit stores (lbrr_step16.cu): sets
// launched = false, launching nothing, where it does not apply (nx not a
// multiple of 16, nx < 64, nx above 1024 (D3Q27, D3Q19) or 2048 (D2Q9), or no
// block fits on an SM).
cudaError_t launch_step_row16(int q, int storage, int model, void *f, const Grid &g, float om1,
                              int parity, int *status, cudaStream_t st, bool &launched);

// The even (parity 0) update of a 16-bit store with direct paired accesses
// (lbrr_pair16.cu); usable when pair16_even_supported(g) (nx a multiple of 64).
bool pair16_even_supported(const Grid &g);
cudaError_t launch_step_pair16_even(int q, int storage, int model, void *f, const Grid &g,
                                    float om1, cudaStream_t st);

// The odd (parity 1) update of a 16-bit store through shared-memory row
// segments (lbrr_step16.cu); usable when tiled16_supported(g) (nx a multiple
// of 128).
bool tiled16_supported(const Grid &g);
cudaError_t launch_step_tiled16_odd(int q, int storage, int model, void *f, const Grid &g,
                                    float om1, cudaStream_t st);

// f = f0 + f1 (mode 1) or f0 (mode 0) from device fields rho [N], u [D][N].
cudaError_t launch_init(int q, int storage, int model, void *f, const Grid &g, const float *rho,
                        const float *u, float tau, int mode, cudaStream_t st);

// Logical shifted populations (natural order) to / from float32 [Q][N].
cudaError_t launch_get_populations(int q, int storage, const void *f, const Grid &g, int parity,
                                   float *dst, cudaStream_t st);
cudaError_t launch_set_populations(int q, int storage, void *f, const Grid &g, const float *src,
                                   cudaStream_t st);

// rho [N], u [D][N], pi1 [3|6][N]; NULL pointers skip the field.
cudaError_t launch_moments(int q, int storage, const void *f, const Grid &g, int parity,
                           float *rho, float *u, float *pi1, cudaStream_t st);

// Deterministic FP64 reduction of (sum drho, sum rho u, 0.5 sum rho |u|^2)
// into partials [nb][kRedValues], nb = min(max_blocks, cells / kRedThreads
// rounded up), then into out[kRedValues]. The summation order depends only
// on the grid and max_blocks, so results repeat bit for bit.
cudaError_t launch_diagnostics(int q, int storage, const void *f, const Grid &g, int parity,
                               int max_blocks, double *partials, double *out, cudaStream_t st);

// 0.5 sum |curl u|^2 from a velocity field u [D][N] (central differences),
// reduced through partials [max_blocks at most] into out[0]. With walls: second-order
// one-sided differences on the wall planes and the trapezoidal weights (1/2
// per wall plane a node lies on).
cudaError_t launch_enstrophy(int d, const float *u, const Grid &g, int max_blocks,
                             double *partials, double *out, cudaStream_t st);

// As launch_diagnostics with the number of partial-sum blocks given by the
// caller (partials must hold nblocks * kRedValues doubles); used by the
// entry point that brings its own scratch.
cudaError_t launch_diagnostics_blocks(int q, int storage, const void *f, const Grid &g,
                                      int parity, int nblocks, double *partials, double *out,
                                      cudaStream_t st);

// One block waiting (bounded, `iterations` try-waits) on an mbarrier nothing
// arrives on; sets *status to 1 when the wait expires (lbrr_selftest.cu).
cudaError_t launch_wait_selftest(unsigned iterations, int *status, cudaStream_t st);

// Records a message for lb_last_error(NULL) on the calling thread.
int report_error(int code, const char *fmt, ...);

}  // namespace lbrr
