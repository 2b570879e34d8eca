/*
 * lbrr.h - C ABI of the GB300 (sm_103a) recursive-regularized BGK lattice
 * Boltzmann library, liblbrr.so.
 *
 * The method is the regularized collide-and-stream update of Malaspinas,
 * arXiv:1505.06900, Sec. 3.5 (eq_discr_bgk_reg):
 *
 *     f_i(x + xi_i, t + 1) = f0_i + (1 - 1/tau) f1_i,
 *
 * where f0 is the equilibrium expanded on the full D2Q9 / D3Q27 Hermite basis
 * (Sec. 3.2, eq_fzero_d2q9 / eq_fzero_d3q27), f1 the off-equilibrium part
 * (eq_fone_d2q9 / eq_fone_d3q27) whose coefficients of order n >= 3 follow
 * from u and a1^(2) = Pi^(1) by the recursion of Sec. 3.1 (eq_rel_a1,
 * Appendix B without the starred terms), and tau is the shifted relaxation
 * time tau-bar of Sec. 3.4 (kinematic viscosity nu = (tau - 1/2) / 3).
 *
 * Conventions shared by every call:
 *  - Lattices: D2Q9 (nz must be 1) and D3Q27. Velocity i has components
 *    (i % 3 - 1, (i / 3) % 3 - 1, i / 9 - 1); the opposite velocity is Q-1-i.
 *    D3Q19, which Sec. 5 names as the cheaper 3-D lattice without defining
 *    its recursion, is the D3Q27 list with the eight corners (|xi|^2 = 3)
 *    left out, in the same order (opposite 18-i again), weights 1/3, 1/18,
 *    1/36. Its quadrature is exact only to total degree five, so its order-3
 *    basis is, for each odd index b with even pair (a, c), H_aab + H_bcc and
 *    H_aab - H_bcc (the largest set of order-3 Hermite sums D3Q19 keeps
 *    orthogonal); f0 and f1 are expanded on 1, xi, H2 and those six, with
 *    the Hermite coefficients of Sec. 2 (f0) and of the recursion eq_rel_a1
 *    (f1). Every call accepts it where it accepts D3Q27, except the learned
 *    closure.
 *  - Fields are structure-of-arrays, x fastest: element (c, z, y, x) of a
 *    field with C components is at ((c * nz + z) * ny + y) * nx + x.
 *  - Populations exchanged with the caller are "shifted": df_i = f_i - w_i,
 *    float32, one array of Q * nx * ny * nz values.
 *  - Pointers documented as device pointers must point to memory of the
 *    context's device (cudaMalloc, torch tensors) or managed memory; the
 *    caller owns them. Each call checks them (cudaPointerGetAttributes,
 *    which allocates nothing) and answers LB_EINVAL, before any kernel runs,
 *    for a host pointer or another device's memory.
 *  - All work is ordered on the context's stream (lb_set_stream); calls that
 *    return values to host memory synchronise that stream.
 *  - Every call returns LB_OK or an error code; on error the context's state
 *    is unchanged unless stated otherwise and lb_last_error() explains it.
 *  - A context is not thread-safe: one host thread at a time.
 */
#ifndef LBRR_H
#define LBRR_H

#if defined(__GNUC__)
#define LB_API __attribute__((visibility("default")))
#else
#define LB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define LB_OK 0
#define LB_EINVAL 1    /* bad argument (lattice, sizes, tau <= 1/2, null pointer ...) */
#define LB_ENOMEM 2    /* a device or host allocation failed */
#define LB_ECUDA 3     /* a CUDA call or kernel launch failed */
#define LB_EDIVERGED 4 /* a diagnostic is not finite: the run has blown up */
#define LB_ETIMEOUT 5  /* a bounded wait inside a kernel expired (its results are incomplete) */

/* lattices */
#define LB_D2Q9 9
#define LB_D3Q19 19 /* D3Q27 without the corners; order-3 sums/differences basis */
#define LB_D3Q27 27

/* storage of the populations in device memory */
#define LB_STORE_F32 0  /* df_i = f_i - w_i as float32 (4 bytes) */
#define LB_STORE_F16 1  /* (f_i - w_i) / w_i as IEEE binary16, round to nearest even */
#define LB_STORE_BF16 2 /* (f_i - w_i) / w_i as bfloat16, round to nearest even */

/* collision models */
#define LB_COLLIDE_RR 0   /* recursive regularized, Sec. 3.5 (the paper's model) */
#define LB_COLLIDE_REG2 1 /* order-2 regularized comparator, Sec. 3.8.1 (eq_feq_2) */
#define LB_COLLIDE_BGK 2  /* plain BGK, f - (f - f0)/tau with the full-basis f0 of Sec. 3.2
                             (eq_full_discr_bgk, Sec. 3.4); initialised like RR */

/* initialisation modes of lb_init_fields */
#define LB_INIT_EQ 0        /* f = f0(rho, u) */
#define LB_INIT_EQ_NEQ_FD 1 /* f = f0 + f1 with a1^(2) = -2 c_s^2 rho tau S, S by periodic
                               central differences of u (Sec. 3.3, constitutive relation) */

typedef struct lb_ctx lb_ctx;

typedef struct lb_options {
  int lattice;    /* LB_D2Q9, LB_D3Q19 or LB_D3Q27 */
  int nx, ny, nz; /* grid size in cells, each >= 1; nz == 1 for D2Q9 */
  double tau;     /* shifted relaxation time tau-bar > 1/2 (Sec. 3.4) */
  int periodic;   /* must be 1: every face without a wall is periodic */
  int storage;    /* LB_STORE_* */
  int collision;  /* LB_COLLIDE_* */
  int walls;      /* LB_WALL_* mask: no-slip walls through the first and last
                     node planes of these axes (each >= 3 nodes), 0 = none */
} lb_options;

/* No-slip walls (Sec. 3.7, boundary conditions): the boundary nodes lie on
 * the walls and carry u = 0; each is closed by the regularized Dirichlet
 * procedure in its zero-velocity form (an unknown population, one that would
 * stream in from outside, takes the value of its opposite, so rho and
 * Pi^(1) follow from the lattice symmetries; a buried link of an edge or
 * corner is set to equilibrium) and then relaxed to f0(rho, 0) +
 * (1 - 1/tau) f1(Pi^(1)) whatever the collision model. lb_moments and
 * lb_diagnostics report these closed states (u = 0 on the walls);
 * lb_enstrophy uses second-order one-sided differences on the wall planes and
 * the trapezoidal rule (weight 1/2 per wall plane a node lies on);
 * lb_init_fields starts wall nodes at rest. Populations that stream in from
 * outside are undefined in lb_get_populations. The learned closure and
 * lb_coarsen need periodic contexts; lb_diagnostics_static assumes one. */
#define LB_WALL_X 1
#define LB_WALL_Y 2
#define LB_WALL_Z 4

/* Create a context holding one device population store of Q*nx*ny*nz values
 * (AA pattern: one buffer, updated in place) on the current CUDA device. The
 * populations start at rest (f = w, rho = 1, u = 0). Storage F32, model RR.
 * Returns LB_EINVAL for a bad lattice, a size < 1, nz != 1 with D2Q9,
 * tau <= 1/2 or periodic != 1; LB_ENOMEM if the store does not fit. No walls.
 * Sec. 3.2 (q populations per node), Sec. 3.4 (tau). */
LB_API int lb_create(lb_ctx **out, int lattice, int nx, int ny, int nz, double tau, int periodic);

/* As lb_create, with the storage precision, collision model and walls
 * chosen; LB_EINVAL also for a walls mask outside the lattice's axes or a
 * walled axis with fewer than 3 nodes. */
LB_API int lb_create_ex(lb_ctx **out, const lb_options *opt);

/* Free the context and its device memory. NULL is accepted. */
LB_API void lb_destroy(lb_ctx *ctx);

/* Text of the last error on this context; with ctx == NULL, of the last
 * failed lb_create/lb_create_ex on the calling thread. Never NULL. */
LB_API const char *lb_last_error(const lb_ctx *ctx);

/* Order all later work of the context on `stream` (a cudaStream_t; NULL is the
 * legacy default stream). */
LB_API int lb_set_stream(lb_ctx *ctx, void *stream);

/* Set the populations from macroscopic fields (device pointers): rho [N],
 * u [D][N], float32. init_mode LB_INIT_EQ or LB_INIT_EQ_NEQ_FD. Resets the
 * step count. Sec. 3.2 (eq_fzero_*), Sec. 3.1 (eq_rel_a1), Sec. 3.3. */
LB_API int lb_init_fields(lb_ctx *ctx, const float *rho, const float *u, int init_mode);

/* Advance n >= 0 full collide-and-stream updates (eq_discr_bgk_reg). n == 0 is
 * a no-op. Asynchronous on the context's stream. Without a learned closure,
 * runs of 8 updates are replayed from a CUDA graph that the context captures
 * on first use (one per starting AA parity, on a stream of its own); the
 * results are those of update-by-update launches, bit for bit. While the
 * context's stream is being captured by the caller, updates are launched one
 * by one into that capture. With a 16-bit store the
 * update waits (boundedly) for its own bulk copies; if such a wait ever
 * expires, the next lb_diagnostics or lb_get_state returns LB_ETIMEOUT. */
LB_API int lb_step(lb_ctx *ctx, int n);

/* Macroscopic fields of the current populations into device buffers:
 * rho [N], u [D][N], pi1 [3 or 6][N] (xx, xy, yy in 2D; xx, xy, xz, yy, yz, zz
 * in 3D) with pi1 = a1^(2) = sum xi xi f - rho c_s^2 I - rho u u (Sec. 2,
 * P^(1) = a1^(2)). Any pointer may be NULL to skip that field. */
LB_API int lb_moments(lb_ctx *ctx, float *rho, float *u, float *pi1);

/* Global diagnostics in double precision into host memory out[2 + D]:
 * mass sum rho, momentum sum rho u (D values), kinetic energy
 * 0.5 sum rho |u|^2. Deterministic (fixed reduction order). Synchronises the
 * stream. Returns LB_EDIVERGED (out still filled) if a value is not finite.
 * Uses a device scratch buffer owned by the context. */
LB_API int lb_diagnostics(lb_ctx *ctx, double *out);

/* Enstrophy 0.5 sum |curl u|^2 with periodic central differences (2D:
 * omega = d_x u_y - d_y u_x; the enstrophy of Sec. 4.1 summed over cells),
 * double precision, into host memory *out. Synchronises the stream. */
LB_API int lb_enstrophy(lb_ctx *ctx, double *out);

/* Copy the current populations, in natural order and shifted form
 * df_i(x) = f_i(x) - w_i, float32, into the device buffer dst [Q][N]. */
LB_API int lb_get_populations(lb_ctx *ctx, float *dst);

/* Replace the populations by the shifted float32 values src [Q][N] (device),
 * rounded to the storage precision. Resets the step count. */
LB_API int lb_set_populations(lb_ctx *ctx, const float *src);

/* Size in bytes of the raw device store (for lb_get_state / lb_set_state). */
LB_API long long lb_state_bytes(const lb_ctx *ctx);

/* Copy the raw store (storage precision, AA slot order) and the step count
 * parity to dst (host or device memory, lb_state_bytes bytes) - a checkpoint.
 * Synchronises the stream. */
LB_API int lb_get_state(lb_ctx *ctx, void *dst, int *parity);

/* Restore a checkpoint written by lb_get_state of a context with the same
 * lattice, size and storage. parity must be 0 or 1. */
LB_API int lb_set_state(lb_ctx *ctx, const void *src, int parity);

/* End-to-end run through host memory: copy rho_h [N] and u_h [D][N] (host,
 * float32; pinned memory makes the copies asynchronous) to the device,
 * initialise with init_mode, advance nsteps, and copy the final rho and u
 * into rho_out_h / u_out_h (host, may be NULL) and the diagnostics of
 * lb_diagnostics into diag_h[2 + D] (host, may be NULL). Synchronises. */
LB_API int lb_run_host(lb_ctx *ctx, const float *rho_h, const float *u_h, int init_mode, int nsteps,
                       float *rho_out_h, float *u_out_h, double *diag_h);

/* Description of a context into out[8]: lattice, nx, ny, nz, storage,
 * collision, number of steps taken, bytes moved per cell update. */
LB_API int lb_info(const lb_ctx *ctx, long long *out);

/* ---------------------------------------------------------------------------
 * Learned closure (an extension around the method; the paper has no learned
 * component). A small network predicts, from the moments (rho - 1, u, Pi1) of
 * a D3Q27 cell and of its 26 periodic neighbours, the off-equilibrium Hermite
 * coefficients of orders 3..6 that the recursion of Sec. 3.1 leaves out of a
 * coarse-grained (2x2x2 box-filtered) fine run; the prediction is added to the
 * recursion's coefficients before the (1 - 1/tau) relaxation of
 * eq_discr_bgk_reg. Zero weights reproduce the RR update exactly.
 *
 * Network: y = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3, x in R^288 (270 used),
 * hidden 64 and 64, y in R^32 (17 used). Parameters are packed as W1 [64][288],
 * b1 [64], W2 [64][64], b2 [64], W3 [32][64], b3 [32] (LB_MLP_PARAMS floats,
 * row-major, W[out][in]). Products run on tensor cores with BF16 operands
 * (weights and activations rounded to BF16) and FP32 accumulation; the master
 * parameters and the Adam state are FP32.
 *
 * Features (BF16 [N][288]): feature 10 * nb + k is moment k of neighbour
 * nb = (dx+1) + 3(dy+1) + 9(dz+1), minus in_mean[k], times in_inv_std[k];
 * 270..287 are zero. Targets (FP32 [N][32]): coefficient k (order xxy, xxz,
 * xyy, xzz, yzz, yyz, xyz, xxyy, xxzz, yyzz, xyzz, xyyz, xxyz, xxyzz, xxyyz,
 * xyyzz, xxyyzz) of f - f_RR divided by out_scale[k]; 17..31 are zero. Loss:
 * mean over rows and the 17 used outputs of (y - t)^2.
 * ------------------------------------------------------------------------- */
#define LB_MLP_PARAMS 24736
#define LB_MLP_IN 288
#define LB_MLP_OUT 32

typedef struct lb_mlp lb_mlp;

/* Network on the current device, parameters zero, Adam state empty, scaling
 * in_mean = 0, in_inv_std = 1, out_scale = 1. */
LB_API int lb_mlp_create(lb_mlp **out);
LB_API void lb_mlp_destroy(lb_mlp *mlp);
LB_API const char *lb_mlp_last_error(const lb_mlp *mlp);
LB_API int lb_mlp_set_stream(lb_mlp *mlp, void *stream);
/* Copy LB_MLP_PARAMS packed floats (host or device memory); resets Adam. */
LB_API int lb_mlp_set_params(lb_mlp *mlp, const float *params);
LB_API int lb_mlp_get_params(lb_mlp *mlp, float *params);
/* Feature and target standardisation (host arrays of 10, 10 and 17 floats;
 * in_inv_std and out_scale must be finite and non-zero). */
LB_API int lb_mlp_set_scaling(lb_mlp *mlp, const float *in_mean, const float *in_inv_std,
                              const float *out_scale);
/* Y [M][32] (device, FP32) = network(X [M][288], device, BF16). Synchronises;
 * LB_ETIMEOUT if a bounded tensor-core wait of the network kernel expired. */
LB_API int lb_mlp_forward(lb_mlp *mlp, const void *X, long long M, float *Y);
/* Gradient of the loss over the batch into grad [LB_MLP_PARAMS] (device) and
 * the loss into *loss (host, may be NULL); parameters unchanged. Deterministic. */
LB_API int lb_mlp_gradients(lb_mlp *mlp, const void *X, const float *T, long long M, float *grad,
                            double *loss);
/* Inspection forms of lb_mlp_forward and lb_mlp_gradients (no counterpart in
 * the paper; they let a test check every layer of the network kernels, not
 * only their end result). They run the same arithmetic and also write, for
 * every row, the FP32 values the kernel computed before it rounded them to
 * BF16 for the next product:
 *   lb_mlp_forward_trace: H [M][128] (device): tanh(W1 x + b1) in columns
 *     0..63, tanh(W2 h1 + b2) in columns 64..127 (h1 rounded to BF16);
 *   lb_mlp_gradients_trace: trace [M][320] (device): h1 (0..63), h2 (64..127),
 *     y (128..159), dy = 2 (y - t) / (17 M) on the used outputs (160..191),
 *     dh2 = (W3^T dy) (1 - h2^2) (192..255, dy rounded to BF16), dh1 =
 *     (W2^T dh2) (1 - h1^2) (256..319, dh2 rounded to BF16).
 * The weight gradients are products of the BF16 roundings of these rows with
 * the BF16 inputs (dW1 = dh1^T x, dW2 = dh2^T h1, dW3 = dy^T h2), the bias
 * gradients sums of the FP32 values (db1 = sum dh1, ...). */
LB_API int lb_mlp_forward_trace(lb_mlp *mlp, const void *X, long long M, float *Y, float *H);
LB_API int lb_mlp_gradients_trace(lb_mlp *mlp, const void *X, const float *T, long long M,
                                  float *grad, double *loss, float *trace);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on the
 * batch; *loss (host, may be NULL) is the loss before the step. With loss
 * NULL the call does not synchronise: if a tensor-core wait of the pass timed
 * out, no parameter changes (nor in later steps) and the next synchronising
 * call on this network returns LB_ETIMEOUT. */
LB_API int lb_mlp_train_step(lb_mlp *mlp, const void *X, const float *T, long long M, float lr,
                             double *loss);
/* Features of every cell of a D3Q27 FP32 RR context into X [N][288] (device). */
LB_API int lb_closure_features(lb_ctx *ctx, const lb_mlp *mlp, void *X);
/* Standardised targets of every cell into T [N][32] (device). */
LB_API int lb_closure_targets(lb_ctx *ctx, const lb_mlp *mlp, float *T);
/* 2x2x2 box average of the populations of `fine` into `coarse` (D3Q27 FP32
 * contexts, fine = 2 x coarse in every direction); resets coarse's step count.
 * The coarse grid of an acoustically scaled run uses tau_c = 1/2 + (tau_f - 1/2)/2. */
LB_API int lb_coarsen(lb_ctx *fine, lb_ctx *coarse);
/* The same with the off-equilibrium part of each averaged cell scaled:
 * f0(rho, u) + neq_scale (fbar - f0(rho, u)), rho and u the moments of the
 * average fbar. With neq_scale = 2 tau_coarse / tau_fine the coarse state
 * carries the off-equilibrium part the coarse grid's own dynamics builds
 * (the constitutive relation a1^(2) = -2 c_s^2 rho tau S of Sec. 3.3 in each
 * grid's lattice units; the strain rate per coarse cell and step is twice the
 * fine one). neq_scale = 1 is lb_coarsen. */
LB_API int lb_coarsen_neq(lb_ctx *fine, lb_ctx *coarse, double neq_scale);
/* Step-matching targets (extension, not in the paper): for two states of the
 * same periodic D3Q27 FP32 RR grid, `pre` at some time and `post` one coarse
 * update later in the reference run (e.g. the filtered fine run two fine
 * steps later), T [N][32] (device) holds per cell the order 3..6 Hermite
 * coefficients of (P - R) / (1 - 1/tau), P_i(x) = post_i(x + xi_i) the
 * populations streaming carries into post, R the RR post-collision of pre
 * (tau of pre), each divided by the network's out_scale and zero padded: the
 * correction that, added to the recursion's coefficients before the
 * relaxation (lb_set_closure), would make the RR update of pre reproduce
 * those coefficients of post. */
LB_API int lb_closure_step_targets(lb_ctx *pre, lb_ctx *post, const lb_mlp *mlp, float *T);
/* Use the network in lb_step (NULL: plain RR). A cell whose standardised
 * prediction exceeds `bound` in magnitude, or whose corrected populations are
 * not all positive, takes the RR update instead and is counted. The network
 * must outlive its use. On grids whose rows are whole 128-cell tiles an
 * update is two kernels: the standardised moments of every cell (BF16), then
 * the tcgen05 network, whose epilogue performs the corrected update of each
 * tile row's cell in place; on other grids the predictions go through device
 * memory to a separate update kernel. If a bounded wait of the network
 * expires (reported as LB_ETIMEOUT), part of the cells of that update were
 * not updated: re-initialise or restore a checkpoint. */
LB_API int lb_set_closure(lb_ctx *ctx, const lb_mlp *mlp, float bound);
/* The same with a dead zone (extension, not in the paper): each standardised
 * prediction y is shrunk to sign(y) max(|y| - dead_zone, 0) before it scales
 * its coefficient, so that predictions at the level of the network's own
 * error leave the cell to plain RR (dead_zone finite and >= 0; 0 is
 * lb_set_closure). The bound applies to the unshrunk prediction. */
LB_API int lb_set_closure_ex(lb_ctx *ctx, const lb_mlp *mlp, float bound, float dead_zone);
/* Inspection form of one closure update (no counterpart in the paper; it lets
 * a test check the fused kernel's network layer by layer): on a context whose
 * learned closure runs the fused row-tile kernel (nx a multiple of 128), one
 * update exactly as lb_step(ctx, 1) performs it, that also writes
 *   trace [N][145] (device, FP32, cells in x-fastest order): the activations
 *     of layers 1 (0..63) and 2 (64..127) before their BF16 rounding and the
 *     17 standardised predictions (128..144) of every cell;
 *   xs_out (device, (nx+2)(ny+2)(nz+2) x 16 BF16): the standardised moments
 *     the update's network read, channels-last with a one-cell periodic halo,
 *     channels 0..9 = rho - 1, u, Pi1 (xx, xy, xz, yy, yz, zz), 10..15 zero.
 * LB_EINVAL on other contexts. */
LB_API int lb_closure_step_trace(lb_ctx *ctx, float *trace, void *xs_out);
/* Cells that fell back to RR since the closure was first set (host out).
 * Synchronises; LB_ETIMEOUT if a bounded tensor-core wait of the closure's
 * network ever expired in lb_step. */
LB_API int lb_closure_fallbacks(lb_ctx *ctx, long long *count);

/* Bounded waits (no counterpart in the paper). Kernels that hand work over
 * with mbarriers (the 16-bit whole-row step, the closure network) give up a
 * wait after a fixed number of try-waits, record it in a device status word
 * and return; the next synchronising call (lb_diagnostics, lb_get_state,
 * lb_closure_fallbacks, lb_mlp_forward ...) reports LB_ETIMEOUT once and
 * clears the word. These calls exist to test that path without faulting a
 * GPU. lb_set_wait_limit / lb_mlp_set_wait_limit set the main-loop limit of
 * a context's / a network's kernels (iterations >= 1; 0 restores the
 * default); waits for copies still in flight after a timeout keep the
 * default. lb_wait_selftest runs one block that waits on an mbarrier nothing
 * arrives on, for `iterations` >= 1 try-waits, and returns LB_ETIMEOUT when
 * the expiry was recorded as it must be (LB_ECUDA otherwise); message in
 * lb_last_error(NULL). */
LB_API int lb_set_wait_limit(lb_ctx *ctx, int iterations);
LB_API int lb_mlp_set_wait_limit(lb_mlp *mlp, int iterations);
LB_API int lb_wait_selftest(int iterations);

/* Largest grid (nx * ny * nz cells) that lb_diagnostics_static accepts. */
#define LB_STATIC_MAX_CELLS 134217728LL /* 512^3 */

/* The diagnostics of lb_diagnostics computed without allocating anything, for
 * callers that cannot call cudaMalloc or cudaFree: those whose device memory
 * is already reserved by another allocator, and those running beside a live
 * simulation that must not take the device-wide synchronisation of cudaFree.
 * The paper has no counterpart; this is a service of the library.
 *
 * store: device pointer to a raw population store of the given lattice, size,
 * storage and AA parity, laid out as lb_get_state writes it; it must be
 * device (or managed) memory of the current device, anything else (a host
 * pointer, another GPU's memory) is rejected with LB_EINVAL. out: host memory,
 * 2 + D doubles (mass, momentum, kinetic energy) as in lb_diagnostics.
 * stream: cudaStream_t to order the work on (NULL: legacy default stream); the
 * call synchronises it. The reduction's partial sums live in a fixed device
 * array inside the library (1.25 MiB per GPU, held until the process exits),
 * so grids above LB_STATIC_MAX_CELLS cells are rejected with LB_EINVAL. All
 * calls on a device share that array: calls that overlap on the GPU race and
 * must be serialised by the caller. The first call on a device (and in each
 * new CUDA context of it) looks up the array's device address
 * (cudaGetSymbolAddress); make it before any stream capture. Errors: LB_EINVAL (bad argument or grid too large), LB_ECUDA,
 * LB_EDIVERGED (out filled, a value is not finite); lb_last_error(NULL) has
 * the text. */
LB_API int lb_diagnostics_static(int lattice, int nx, int ny, int nz, int storage, int parity,
                                 const void *store, double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LBRR_H */
