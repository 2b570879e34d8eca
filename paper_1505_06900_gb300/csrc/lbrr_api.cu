// C ABI of liblbrr.so (declared in include/lbrr.h): context management,
// argument validation, error reporting and the ordering of kernel launches on
// the context's stream. No arithmetic of the method lives here.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "lbrr.h"
#include "lbrr_launch.h"
#include "lbrr_mlp.h"

struct lb_ctx {
  int lattice = 0, d = 0, q = 0;
  lbrr::Grid g{};
  double tau = 0.0;
  int storage = LB_STORE_F32, collision = LB_COLLIDE_RR;
  int parity = 0;          // AA parity: 0 natural order, 1 after an odd number of updates
  long long steps = 0;     // updates since the last (re)initialisation
  int device = 0;
  size_t elem = 4;         // bytes per stored population
  void *f = nullptr;       // population store, q * n elements
  int red_blocks = 0;          // partial-sum blocks: kRedBlocksPerSm x the device's SMs
  double *partials = nullptr;  // reduction scratch, red_blocks * kRedValues doubles
  double *dout = nullptr;      // reduction result, kRedValues doubles
  int *status = nullptr;       // [0] set to 1 by the 16-bit row kernel if a bounded wait
                               // expired (cleared when reported), [1] its main-loop wait limit
  float *fields = nullptr;     // lazily allocated (1 + d) * n floats for enstrophy / run_host
  float *mom = nullptr;        // lazily allocated 10 * n floats: moment field of the closure
  float *ystd = nullptr;       // lazily allocated 17 * n floats: the network's predictions
                               // (grids the fused TMA-fed network does not take)
  void *xs = nullptr;          // feature source of the TMA-fed network (row-tile grids)
  CUtensorMap xs_map{};        // its tensor map
  const lb_mlp *closure = nullptr;  // learned closure in use (not owned)
  float closure_bound = 0.f;
  float closure_dead_zone = 0.f;
  unsigned long long *fallbacks = nullptr;  // device counter of cells that fell back to RR
  cudaStream_t stream = nullptr;
  // CUDA graphs of kGraphSteps plain updates starting at parity 0 / 1 (built
  // on first use, on a private capture stream, and replayed on `stream`)
  cudaStream_t capture = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  bool graph_off = false;  // capture failed once: launch update by update
  char err[512] = {0};
};

struct lb_mlp {
  lbrr::MlpDevice d{};
  float *scaling = nullptr;    // device: in_mean[10], in_inv_std[10], out_scale[17]
  float *gpart = nullptr;      // per-block gradient partials
  float *lpart = nullptr;      // per-block loss partials
  double *dloss = nullptr;
  int *status = nullptr;       // [0] set to 1 by a tensor-core kernel if a wait timed out
                               // (cleared when reported), [1] main-loop wait limit (0 default)
  int nblocks = 0;             // blocks of the training kernel (one per SM)
  long long t = 0;             // Adam steps taken
  int device = 0;
  cudaStream_t stream = nullptr;
  char err[512] = {0};
};

namespace {

thread_local char g_create_err[512] = "no error";

int fail(lb_ctx *c, int code, const char *fmt, ...) {
  char *buf = c ? c->err : g_create_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, 512, fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(lb_ctx *c, cudaError_t e, const char *what) {
  return fail(c, LB_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define LB_CHECK_CTX(c)                                         \
  do {                                                          \
    if (!(c)) return fail(nullptr, LB_EINVAL, "null context");  \
  } while (0)

// NVTX range around an entry point (shown by nsys and other tracing tools;
// free when no tool is attached).
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

// Make the context's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Whether p is memory that device dev can use as its own: device memory of
// dev, or managed memory (cudaPointerGetAttributes allocates nothing).
bool usable_on(const void *p, int dev) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == dev);
}

// LB_OK, or LB_EINVAL naming the argument when p is not usable on the
// context's device; null pointers are left to the caller's own checks.
int need_device(lb_ctx *c, const void *p, const char *what) {
  if (!p || usable_on(p, c->device)) return LB_OK;
  return fail(c, LB_EINVAL, "%s must be device memory of device %d (got a host pointer or "
              "another device's memory)", what, c->device);
}

#define LB_NEED_DEVICE(c, p)                   \
  do {                                         \
    const int rc_ = need_device((c), (p), #p); \
    if (rc_ != LB_OK) return rc_;              \
  } while (0)

int free_all(lb_ctx *c) {
  for (auto &ge : c->graph)
    if (ge) cudaGraphExecDestroy(ge);
  c->graph[0] = c->graph[1] = nullptr;
  if (c->capture) cudaStreamDestroy(c->capture);
  c->capture = nullptr;
  if (c->f) cudaFree(c->f);
  if (c->partials) cudaFree(c->partials);
  if (c->dout) cudaFree(c->dout);
  if (c->status) cudaFree(c->status);
  c->status = nullptr;
  if (c->fields) cudaFree(c->fields);
  if (c->mom) cudaFree(c->mom);
  if (c->ystd) cudaFree(c->ystd);
  if (c->xs) cudaFree(c->xs);
  c->xs = nullptr;
  if (c->fallbacks) cudaFree(c->fallbacks);
  c->mom = nullptr;
  c->ystd = nullptr;
  c->fallbacks = nullptr;
  c->f = nullptr;
  c->partials = nullptr;
  c->dout = nullptr;
  c->fields = nullptr;
  return 0;
}

int ensure_fields(lb_ctx *c) {
  if (c->fields) return LB_OK;
  cudaError_t e = cudaMalloc(&c->fields, sizeof(float) * (size_t)(1 + c->d) * (size_t)c->g.n);
  if (e != cudaSuccess) {
    c->fields = nullptr;
    cudaGetLastError();
    return fail(c, LB_ENOMEM, "cannot allocate %lld bytes of field scratch",
                (long long)(sizeof(float) * (size_t)(1 + c->d) * (size_t)c->g.n));
  }
  return LB_OK;
}

// Deterministic FP64 diagnostics into host out[2 + d].
int diagnostics(lb_ctx *c, double *out) {
  cudaError_t e = lbrr::launch_diagnostics(c->q, c->storage, c->f, c->g, c->parity,
                                           c->red_blocks, c->partials, c->dout, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "diagnostics launch");
  double h[lbrr::kRedValues];
  int st = 0;
  e = cudaMemcpyAsync(h, c->dout, sizeof h, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&st, c->status, sizeof st, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "diagnostics copy");
  if (st) {
    cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
    return fail(c, LB_ETIMEOUT, "a bulk-copy wait of the 16-bit step kernel timed out");
  }
  out[0] = (double)c->g.n + h[0];
  for (int a = 0; a < c->d; ++a) out[1 + a] = h[1 + a];
  out[1 + c->d] = h[4];
  for (int k = 0; k < 2 + c->d; ++k)
    if (!std::isfinite(out[k])) return fail(c, LB_EDIVERGED, "diagnostic %d is not finite", k);
  return LB_OK;
}

}  // namespace

namespace lbrr {
int report_error(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_create_err, sizeof g_create_err, fmt, ap);
  va_end(ap);
  return code;
}
}  // namespace lbrr

extern "C" {

int lb_create_ex(lb_ctx **out, const lb_options *opt) {
  if (!out || !opt) return fail(nullptr, LB_EINVAL, "null argument");
  *out = nullptr;
  const int lat = opt->lattice;
  if (lat != LB_D2Q9 && lat != LB_D3Q19 && lat != LB_D3Q27)
    return fail(nullptr, LB_EINVAL, "unknown lattice %d", lat);
  if (opt->nx < 1 || opt->ny < 1 || opt->nz < 1)
    return fail(nullptr, LB_EINVAL, "grid sizes must be >= 1 (got %d x %d x %d)", opt->nx, opt->ny,
                opt->nz);
  if (lat == LB_D2Q9 && opt->nz != 1) return fail(nullptr, LB_EINVAL, "D2Q9 needs nz == 1");
  if (opt->ny > 65535 || opt->nz > 65535)
    return fail(nullptr, LB_EINVAL, "ny and nz must be <= 65535");
  if (!(opt->tau > 0.5) || !std::isfinite(opt->tau))
    return fail(nullptr, LB_EINVAL, "tau must be a finite number > 1/2 (got %g)", opt->tau);
  if (opt->periodic != 1)
    return fail(nullptr, LB_EINVAL, "periodic must be 1 (the faces without walls are periodic)");
  const int dims = lat == LB_D2Q9 ? 2 : 3;
  if (opt->walls < 0 || opt->walls >= (1 << dims))
    return fail(nullptr, LB_EINVAL, "walls must be a mask of the %d axes (got %d)", dims,
                opt->walls);
  {
    const int sz[3] = {opt->nx, opt->ny, opt->nz};
    for (int a = 0; a < dims; ++a)
      if (((opt->walls >> a) & 1) && sz[a] < 3)
        return fail(nullptr, LB_EINVAL, "a walled axis needs at least 3 nodes");
  }
  if (opt->storage < LB_STORE_F32 || opt->storage > LB_STORE_BF16)
    return fail(nullptr, LB_EINVAL, "unknown storage %d", opt->storage);
  if (opt->collision != LB_COLLIDE_RR && opt->collision != LB_COLLIDE_REG2 &&
      opt->collision != LB_COLLIDE_BGK)
    return fail(nullptr, LB_EINVAL, "unknown collision model %d", opt->collision);
  const long long n = (long long)opt->nx * opt->ny * opt->nz;
  if (n > (1LL << 40)) return fail(nullptr, LB_EINVAL, "grid too large");

  lb_ctx *c = new (std::nothrow) lb_ctx;
  if (!c) return fail(nullptr, LB_ENOMEM, "host allocation failed");
  c->lattice = lat;
  c->q = lat;
  c->d = lat == LB_D2Q9 ? 2 : 3;
  c->g = lbrr::Grid{opt->nx, opt->ny, opt->nz, n, opt->walls};
  c->tau = opt->tau;
  c->storage = opt->storage;
  c->collision = opt->collision;
  c->elem = opt->storage == LB_STORE_F32 ? 4 : 2;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) {
    delete c;
    return fail(nullptr, LB_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
  }
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess || sms < 1) {
    delete c;
    return fail(nullptr, LB_ECUDA, "cannot query the SM count: %s", cudaGetErrorString(e));
  }
  c->red_blocks = lbrr::kRedBlocksPerSm * sms;
  const size_t bytes = c->elem * (size_t)c->q * (size_t)n;
  e = cudaMalloc(&c->f, bytes);
  if (e == cudaSuccess)
    e = cudaMalloc(&c->partials, sizeof(double) * (size_t)c->red_blocks * lbrr::kRedValues);
  if (e == cudaSuccess) e = cudaMalloc(&c->dout, sizeof(double) * lbrr::kRedValues);
  if (e == cudaSuccess) e = cudaMalloc(&c->status, 2 * sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_all(c);
    delete c;
    return fail(nullptr, LB_ENOMEM, "cannot allocate %zu bytes of population store", bytes);
  }
  // rest state: df = 0 in every storage precision
  e = cudaMemset(c->f, 0, bytes);
  if (e == cudaSuccess) e = cudaMemset(c->status, 0, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_all(c);
    delete c;
    return fail(nullptr, LB_ECUDA, "initial clear failed: %s", cudaGetErrorString(e));
  }
  *out = c;
  return LB_OK;
}

int lb_create(lb_ctx **out, int lattice, int nx, int ny, int nz, double tau, int periodic) {
  lb_options o{lattice, nx, ny, nz, tau, periodic, LB_STORE_F32, LB_COLLIDE_RR, 0};
  return lb_create_ex(out, &o);
}

void lb_destroy(lb_ctx *c) {
  if (!c) return;
  DeviceGuard dg(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
}

const char *lb_last_error(const lb_ctx *c) { return c ? c->err : g_create_err; }

int lb_set_stream(lb_ctx *c, void *stream) {
  LB_CHECK_CTX(c);
  c->stream = static_cast<cudaStream_t>(stream);
  return LB_OK;
}

int lb_init_fields(lb_ctx *c, const float *rho, const float *u, int init_mode) {
  Range nvtx_range("lb_init_fields");
  LB_CHECK_CTX(c);
  if (!rho || !u) return fail(c, LB_EINVAL, "rho and u must be device pointers");
  if (init_mode != LB_INIT_EQ && init_mode != LB_INIT_EQ_NEQ_FD)
    return fail(c, LB_EINVAL, "unknown init mode %d", init_mode);
  LB_NEED_DEVICE(c, rho);
  LB_NEED_DEVICE(c, u);
  DeviceGuard dg(c->device);
  cudaError_t e = lbrr::launch_init(c->q, c->storage, c->collision, c->f, c->g, rho, u,
                                    (float)c->tau, init_mode, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "init launch");
  c->parity = 0;
  c->steps = 0;
  return LB_OK;
}

namespace {

// Updates per CUDA graph of plain (closure-free) updates; even, so a replay
// leaves the AA parity as it found it.
constexpr int kGraphSteps = 8;

// The graph of kGraphSteps updates from the context's current parity, built
// once: the same launches as the update-by-update path, recorded by stream
// capture. Null (and never tried again) if the capture fails.
cudaGraphExec_t step_graph(lb_ctx *c, float om1) {
  const int p = c->parity;
  if (c->graph[p] || c->graph_off) return c->graph[p];
  cudaError_t e = cudaSuccess;
  if (!c->capture) e = cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking);
  cudaGraph_t graph = nullptr;
  if (e == cudaSuccess) e = cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < kGraphSteps && le == cudaSuccess; ++k)
      le = lbrr::launch_step(c->q, c->storage, c->collision, c->f, c->g, om1, p ^ (k & 1),
                             c->status, c->capture);
    e = cudaStreamEndCapture(c->capture, &graph);
    if (e == cudaSuccess) e = le;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph[p], graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->graph[p] = nullptr;
    c->graph_off = true;
  }
  return c->graph[p];
}

}  // namespace

int lb_step(lb_ctx *c, int n) {
  Range nvtx_range("lb_step");
  LB_CHECK_CTX(c);
  if (n < 0) return fail(c, LB_EINVAL, "negative step count %d", n);
  DeviceGuard dg(c->device);
  const float om1 = (float)(1.0 - 1.0 / c->tau);
  // runs of plain updates replay a captured graph (one launch per
  // kGraphSteps updates instead of one per update); not while the caller is
  // capturing the context's stream into a graph of its own
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const bool capturing = cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess ||
                         cs != cudaStreamCaptureStatusNone;
  if (capturing) cudaGetLastError();
  while (!c->closure && !capturing && n >= kGraphSteps) {
    cudaGraphExec_t ge = step_graph(c, om1);
    if (!ge) break;
    cudaError_t e = cudaGraphLaunch(ge, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "step graph launch");
    c->steps += kGraphSteps;
    n -= kGraphSteps;
  }
  for (int k = 0; k < n; ++k) {
    cudaError_t e;
    if (c->closure && c->xs) {
      e = lbrr::launch_feature_source(c->closure->d, static_cast<const float *>(c->f), c->g,
                                      c->parity, c->xs, c->stream);
      if (e == cudaSuccess)
        e = lbrr::launch_mlp_conv_step(c->closure->d, c->xs_map, c->g, static_cast<float *>(c->f),
                                       om1, c->parity, c->fallbacks, c->closure_bound,
                                       c->closure_dead_zone,
                                       c->closure->status, c->closure->nblocks, c->stream);
    } else if (c->closure) {
      e = lbrr::launch_moment_field(c->storage, c->f, c->g, c->parity, c->mom, c->stream);
      if (e == cudaSuccess)
        e = lbrr::launch_mlp_tc(c->closure->d, nullptr, c->mom, &c->g, c->g.n, c->ystd,
                                c->closure->status, c->closure->nblocks, c->stream);
      if (e == cudaSuccess)
        e = lbrr::launch_step_delta(c->closure->d, static_cast<float *>(c->f), c->g, om1,
                                    c->parity, c->ystd, c->fallbacks, c->closure_bound,
                                    c->closure_dead_zone,
                                    c->stream);
    } else {
      e = lbrr::launch_step(c->q, c->storage, c->collision, c->f, c->g, om1, c->parity,
                            c->status, c->stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "step launch");
    c->parity ^= 1;
    ++c->steps;
  }
  return LB_OK;
}

int lb_moments(lb_ctx *c, float *rho, float *u, float *pi1) {
  Range nvtx_range("lb_moments");
  LB_CHECK_CTX(c);
  if (!rho && !u && !pi1) return LB_OK;
  LB_NEED_DEVICE(c, rho);
  LB_NEED_DEVICE(c, u);
  LB_NEED_DEVICE(c, pi1);
  DeviceGuard dg(c->device);
  cudaError_t e =
      lbrr::launch_moments(c->q, c->storage, c->f, c->g, c->parity, rho, u, pi1, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "moments launch");
  return LB_OK;
}

int lb_diagnostics(lb_ctx *c, double *out) {
  Range nvtx_range("lb_diagnostics");
  LB_CHECK_CTX(c);
  if (!out) return fail(c, LB_EINVAL, "null output");
  DeviceGuard dg(c->device);
  return diagnostics(c, out);
}

int lb_enstrophy(lb_ctx *c, double *out) {
  Range nvtx_range("lb_enstrophy");
  LB_CHECK_CTX(c);
  if (!out) return fail(c, LB_EINVAL, "null output");
  DeviceGuard dg(c->device);
  int rc = ensure_fields(c);
  if (rc != LB_OK) return rc;
  float *u = c->fields + c->g.n;
  cudaError_t e = lbrr::launch_moments(c->q, c->storage, c->f, c->g, c->parity, nullptr, u,
                                       nullptr, c->stream);
  if (e == cudaSuccess) e = lbrr::launch_enstrophy(c->d, u, c->g, c->red_blocks, c->partials,
                                                    c->dout, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, c->dout, sizeof(double), cudaMemcpyDeviceToHost,
                                            c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "enstrophy");
  if (!std::isfinite(*out)) return fail(c, LB_EDIVERGED, "enstrophy is not finite");
  return LB_OK;
}

int lb_get_populations(lb_ctx *c, float *dst) {
  LB_CHECK_CTX(c);
  if (!dst) return fail(c, LB_EINVAL, "null destination");
  LB_NEED_DEVICE(c, dst);
  DeviceGuard dg(c->device);
  cudaError_t e =
      lbrr::launch_get_populations(c->q, c->storage, c->f, c->g, c->parity, dst, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "get_populations launch");
  return LB_OK;
}

int lb_set_populations(lb_ctx *c, const float *src) {
  LB_CHECK_CTX(c);
  if (!src) return fail(c, LB_EINVAL, "null source");
  LB_NEED_DEVICE(c, src);
  DeviceGuard dg(c->device);
  cudaError_t e = lbrr::launch_set_populations(c->q, c->storage, c->f, c->g, src, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "set_populations launch");
  c->parity = 0;
  c->steps = 0;
  return LB_OK;
}

long long lb_state_bytes(const lb_ctx *c) {
  return c ? (long long)(c->elem * (size_t)c->q * (size_t)c->g.n) : -1;
}

int lb_get_state(lb_ctx *c, void *dst, int *parity) {
  Range nvtx_range("lb_get_state");
  LB_CHECK_CTX(c);
  if (!dst || !parity) return fail(c, LB_EINVAL, "null argument");
  DeviceGuard dg(c->device);
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(dst, c->f, (size_t)lb_state_bytes(c), cudaMemcpyDefault,
                                  c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&st, c->status, sizeof st, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "get_state copy");
  if (st) {
    cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
    return fail(c, LB_ETIMEOUT, "a bulk-copy wait of the 16-bit step kernel timed out");
  }
  *parity = c->parity;
  return LB_OK;
}

int lb_set_state(lb_ctx *c, const void *src, int parity) {
  Range nvtx_range("lb_set_state");
  LB_CHECK_CTX(c);
  if (!src) return fail(c, LB_EINVAL, "null source");
  if (parity != 0 && parity != 1) return fail(c, LB_EINVAL, "parity must be 0 or 1");
  DeviceGuard dg(c->device);
  cudaError_t e = cudaMemcpyAsync(c->f, src, (size_t)lb_state_bytes(c), cudaMemcpyDefault,
                                  c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "set_state copy");
  c->parity = parity;
  c->steps = parity;
  return LB_OK;
}

int lb_run_host(lb_ctx *c, const float *rho_h, const float *u_h, int init_mode, int nsteps,
                float *rho_out_h, float *u_out_h, double *diag_h) {
  Range nvtx_range("lb_run_host");
  LB_CHECK_CTX(c);
  if (!rho_h || !u_h) return fail(c, LB_EINVAL, "rho and u must be host pointers");
  if (nsteps < 0) return fail(c, LB_EINVAL, "negative step count");
  if (init_mode != LB_INIT_EQ && init_mode != LB_INIT_EQ_NEQ_FD)
    return fail(c, LB_EINVAL, "unknown init mode %d", init_mode);
  DeviceGuard dg(c->device);
  int rc = ensure_fields(c);
  if (rc != LB_OK) return rc;
  const size_t nb = sizeof(float) * (size_t)c->g.n;
  float *rho_d = c->fields, *u_d = c->fields + c->g.n;
  cudaError_t e = cudaMemcpyAsync(rho_d, rho_h, nb, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(u_d, u_h, nb * c->d, cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "run_host upload");
  rc = lb_init_fields(c, rho_d, u_d, init_mode);
  if (rc == LB_OK) rc = lb_step(c, nsteps);
  if (rc != LB_OK) return rc;
  if (rho_out_h || u_out_h) {
    rc = lb_moments(c, rho_d, u_d, nullptr);
    if (rc != LB_OK) return rc;
    if (rho_out_h) e = cudaMemcpyAsync(rho_out_h, rho_d, nb, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && u_out_h)
      e = cudaMemcpyAsync(u_out_h, u_d, nb * c->d, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "run_host download");
  }
  if (diag_h) return diagnostics(c, diag_h);
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "run_host");
  return LB_OK;
}

int lb_info(const lb_ctx *c, long long *out) {
  if (!c || !out) return LB_EINVAL;
  out[0] = c->lattice;
  out[1] = c->g.nx;
  out[2] = c->g.ny;
  out[3] = c->g.nz;
  out[4] = c->storage;
  out[5] = c->collision;
  out[6] = c->steps;
  out[7] = 2LL * c->q * (long long)c->elem;
  return LB_OK;
}

// ------------------------------------------------------------ learned closure

static int mlp_fail(lb_mlp *m, int code, const char *fmt, ...) {
  char *buf = m ? m->err : nullptr;
  va_list ap;
  va_start(ap, fmt);
  if (buf)
    vsnprintf(buf, 512, fmt, ap);
  va_end(ap);
  return code;
}

// LB_OK, or LB_EINVAL naming the argument when p is not usable on the
// network's device; null pointers are left to the caller's own checks.
static int mlp_need_device(lb_mlp *m, const void *p, const char *what) {
  if (!p || usable_on(p, m->device)) return LB_OK;
  return mlp_fail(m, LB_EINVAL, "%s must be device memory of device %d (got a host pointer or "
                  "another device's memory)", what, m->device);
}

#define LB_MLP_NEED_DEVICE(m, p)                   \
  do {                                             \
    const int rc_ = mlp_need_device((m), (p), #p); \
    if (rc_ != LB_OK) return rc_;                  \
  } while (0)

void lb_mlp_destroy(lb_mlp *m) {
  if (!m) return;
  DeviceGuard dg(m->device);
  if (m->stream) cudaStreamSynchronize(m->stream);
  void *bufs[] = {m->d.params, m->d.adam_m, m->d.adam_v, m->d.w1,    m->d.w2,
                  m->d.w3,     m->d.w2t,    m->d.w3t,    m->scaling, m->gpart,
                  m->lpart,    m->dloss,    m->status};
  for (void *b : bufs)
    if (b) cudaFree(b);
  delete m;
}

int lb_mlp_create(lb_mlp **out) {
  if (!out) return fail(nullptr, LB_EINVAL, "null argument");
  *out = nullptr;
  lb_mlp *m = new (std::nothrow) lb_mlp;
  if (!m) return fail(nullptr, LB_ENOMEM, "host allocation failed");
  cudaError_t e = cudaGetDevice(&m->device);
  if (e != cudaSuccess) {
    delete m;
    return fail(nullptr, LB_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device);
  m->nblocks = sms > 0 ? sms : 1;
  const size_t P = lbrr::kMlpParams;
  e = cudaMalloc(&m->d.params, 4 * P);
  if (e == cudaSuccess) e = cudaMalloc(&m->d.adam_m, 4 * P);
  if (e == cudaSuccess) e = cudaMalloc(&m->d.adam_v, 4 * P);
  if (e == cudaSuccess) e = cudaMalloc(&m->d.w1, 2 * lbrr::kMlpHidden * lbrr::kMlpIn);
  if (e == cudaSuccess) e = cudaMalloc(&m->d.w2, 2 * lbrr::kMlpHidden * lbrr::kMlpHidden);
  if (e == cudaSuccess) e = cudaMalloc(&m->d.w3, 2 * lbrr::kMlpOut * lbrr::kMlpHidden);
  if (e == cudaSuccess) e = cudaMalloc(&m->d.w2t, 2 * lbrr::kMlpHidden * lbrr::kMlpHidden);
  if (e == cudaSuccess) e = cudaMalloc(&m->d.w3t, 2 * lbrr::kMlpOut * lbrr::kMlpHidden);
  if (e == cudaSuccess) e = cudaMalloc(&m->scaling, 4 * 37);
  if (e == cudaSuccess) e = cudaMalloc(&m->gpart, 4 * P * (size_t)m->nblocks);
  if (e == cudaSuccess) e = cudaMalloc(&m->lpart, 4 * (size_t)m->nblocks);
  if (e == cudaSuccess) e = cudaMalloc(&m->dloss, sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&m->status, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(m->status, 0, 2 * sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    lb_mlp_destroy(m);
    return fail(nullptr, LB_ENOMEM, "cannot allocate the network");
  }
  m->d.b1 = m->d.params + lbrr::kOffB1;
  m->d.b2 = m->d.params + lbrr::kOffB2;
  m->d.b3 = m->d.params + lbrr::kOffB3;
  m->d.in_mean = m->scaling;
  m->d.in_inv_std = m->scaling + 10;
  m->d.out_scale = m->scaling + 20;
  float sc[37];
  for (int k = 0; k < 37; ++k) sc[k] = k < 10 ? 0.f : 1.f;
  e = cudaMemset(m->d.params, 0, 4 * P);
  if (e == cudaSuccess) e = cudaMemset(m->d.adam_m, 0, 4 * P);
  if (e == cudaSuccess) e = cudaMemset(m->d.adam_v, 0, 4 * P);
  if (e == cudaSuccess) e = cudaMemcpy(m->scaling, sc, sizeof sc, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = lbrr::launch_mlp_refresh(m->d, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    lb_mlp_destroy(m);
    return fail(nullptr, LB_ECUDA, "network initialisation failed: %s", cudaGetErrorString(e));
  }
  *out = m;
  return LB_OK;
}

const char *lb_mlp_last_error(const lb_mlp *m) { return m ? m->err : g_create_err; }

int lb_mlp_set_stream(lb_mlp *m, void *stream) {
  if (!m) return fail(nullptr, LB_EINVAL, "null network");
  m->stream = static_cast<cudaStream_t>(stream);
  return LB_OK;
}

int lb_mlp_set_params(lb_mlp *m, const float *params) {
  if (!m || !params) return mlp_fail(m, LB_EINVAL, "null argument");
  DeviceGuard dg(m->device);
  const size_t bytes = 4 * (size_t)lbrr::kMlpParams;
  cudaError_t e = cudaMemcpyAsync(m->d.params, params, bytes, cudaMemcpyDefault, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->d.adam_m, 0, bytes, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->d.adam_v, 0, bytes, m->stream);
  if (e == cudaSuccess) e = lbrr::launch_mlp_refresh(m->d, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return mlp_fail(m, LB_ECUDA, "set_params: %s", cudaGetErrorString(e));
  m->t = 0;
  return LB_OK;
}

// LB_ETIMEOUT if a tensor-core wait of the network ever timed out (synchronises).
static int mlp_status(lb_mlp *m, cudaStream_t st) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, m->status, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return mlp_fail(m, LB_ECUDA, "status: %s", cudaGetErrorString(e));
  if (h) {
    cudaMemsetAsync(m->status, 0, sizeof(int), st);
    return mlp_fail(m, LB_ETIMEOUT, "a tensor-core wait of the network timed out");
  }
  return LB_OK;
}

int lb_mlp_get_params(lb_mlp *m, float *params) {
  if (!m || !params) return mlp_fail(m, LB_EINVAL, "null argument");
  DeviceGuard dg(m->device);
  cudaError_t e = cudaMemcpyAsync(params, m->d.params, 4 * (size_t)lbrr::kMlpParams,
                                  cudaMemcpyDefault, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return mlp_fail(m, LB_ECUDA, "get_params: %s", cudaGetErrorString(e));
  return mlp_status(m, m->stream);
}

int lb_mlp_set_scaling(lb_mlp *m, const float *in_mean, const float *in_inv_std,
                       const float *out_scale) {
  if (!m || !in_mean || !in_inv_std || !out_scale) return mlp_fail(m, LB_EINVAL, "null argument");
  float sc[37];
  std::memcpy(sc, in_mean, 40);
  std::memcpy(sc + 10, in_inv_std, 40);
  std::memcpy(sc + 20, out_scale, 68);
  for (int k = 0; k < 37; ++k)
    if (!std::isfinite(sc[k]) || (k >= 10 && sc[k] == 0.f))
      return mlp_fail(m, LB_EINVAL, "scaling value %d is zero or not finite", k);
  DeviceGuard dg(m->device);
  cudaError_t e = cudaMemcpyAsync(m->scaling, sc, sizeof sc, cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return mlp_fail(m, LB_ECUDA, "set_scaling: %s", cudaGetErrorString(e));
  return LB_OK;
}

static int mlp_forward(lb_mlp *m, const void *X, long long M, float *Y, float *H) {
  if (!m || !X || !Y || M < 1) return mlp_fail(m, LB_EINVAL, "bad argument");
  LB_MLP_NEED_DEVICE(m, X);
  LB_MLP_NEED_DEVICE(m, Y);
  LB_MLP_NEED_DEVICE(m, H);
  DeviceGuard dg(m->device);
  cudaError_t e =
      lbrr::launch_mlp_tc(m->d, X, nullptr, nullptr, M, Y, m->status, m->nblocks, m->stream, H);
  if (e != cudaSuccess) return mlp_fail(m, LB_ECUDA, "forward: %s", cudaGetErrorString(e));
  return mlp_status(m, m->stream);
}

int lb_mlp_forward(lb_mlp *m, const void *X, long long M, float *Y) {
  return mlp_forward(m, X, M, Y, nullptr);
}

int lb_mlp_forward_trace(lb_mlp *m, const void *X, long long M, float *Y, float *H) {
  if (!H) return mlp_fail(m, LB_EINVAL, "null activation buffer");
  return mlp_forward(m, X, M, Y, H);
}

static int mlp_backward(lb_mlp *m, const void *X, const float *T, long long M, float *grad,
                        int adam, float lr, double *loss, float *trace = nullptr) {
  if (!m || !X || !T || M < 1) return mlp_fail(m, LB_EINVAL, "bad argument");
  LB_MLP_NEED_DEVICE(m, X);
  LB_MLP_NEED_DEVICE(m, T);
  LB_MLP_NEED_DEVICE(m, grad);
  LB_MLP_NEED_DEVICE(m, trace);
  if (adam && !(lr > 0.f && std::isfinite(lr)))
    return mlp_fail(m, LB_EINVAL, "learning rate must be positive");
  DeviceGuard dg(m->device);
  const long long tiles = (M + lbrr::kMlpTrainRows - 1) / lbrr::kMlpTrainRows;
  const int nb = (int)(tiles < m->nblocks ? tiles : m->nblocks);
  cudaError_t e = lbrr::launch_mlp_train(m->d, X, T, M, m->gpart, m->lpart, m->status, nb,
                                         m->stream, trace);
  float bc1 = 1.f, bc2 = 1.f;
  if (adam) {
    const long long t = m->t + 1;
    bc1 = (float)(1.0 - std::pow(0.9, (double)t));
    bc2 = (float)(1.0 - std::pow(0.999, (double)t));
  }
  if (e == cudaSuccess)
    e = lbrr::launch_mlp_reduce(m->d, m->gpart, nb, grad, adam, lr, bc1, bc2, m->lpart,
                                loss ? m->dloss : nullptr, m->status, m->stream);
  if (e == cudaSuccess && loss) {
    double h = 0.0;
    e = cudaMemcpyAsync(&h, m->dloss, sizeof h, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    *loss = h / ((double)M * lbrr::kMlpOutUsed);
  }
  if (e != cudaSuccess) return mlp_fail(m, LB_ECUDA, "backward: %s", cudaGetErrorString(e));
  // A pass whose wait timed out changes no parameter (the Adam kernel checks
  // the status word on the device). Calls that synchronise anyway (a loss was
  // asked for) report it here; otherwise the next synchronising call does.
  if (loss || !adam) {
    const int rc = mlp_status(m, m->stream);
    if (rc != LB_OK) return rc;
  }
  if (adam) ++m->t;
  return LB_OK;
}

int lb_mlp_gradients(lb_mlp *m, const void *X, const float *T, long long M, float *grad,
                     double *loss) {
  if (!grad) return mlp_fail(m, LB_EINVAL, "null gradient buffer");
  return mlp_backward(m, X, T, M, grad, 0, 0.f, loss);
}

int lb_mlp_gradients_trace(lb_mlp *m, const void *X, const float *T, long long M, float *grad,
                           double *loss, float *trace) {
  if (!grad || !trace) return mlp_fail(m, LB_EINVAL, "null gradient or trace buffer");
  return mlp_backward(m, X, T, M, grad, 0, 0.f, loss, trace);
}

int lb_mlp_train_step(lb_mlp *m, const void *X, const float *T, long long M, float lr,
                      double *loss) {
  Range nvtx_range("lb_mlp_train_step");
  return mlp_backward(m, X, T, M, nullptr, 1, lr, loss);
}

// Closure scratch: the moment field (features of lb_closure_features and the
// network of grids that are not whole row tiles), the predictions, and for
// row-tile grids the feature source of the TMA-fed network with its map.
static int ensure_mom(lb_ctx *c, bool for_step) {
  const bool conv = for_step && lbrr::mlp_conv_supported(c->g);
  cudaError_t e = cudaSuccess;
  if (!conv && !c->mom) e = cudaMalloc(&c->mom, sizeof(float) * 10 * (size_t)c->g.n);
  if (e == cudaSuccess && !conv && !c->ystd)  // the fused network writes no predictions
    e = cudaMalloc(&c->ystd, sizeof(float) * 17 * (size_t)c->g.n);
  if (e == cudaSuccess && conv && !c->xs) {
    e = cudaMalloc(&c->xs, lbrr::feature_source_bytes(c->g));
    if (e == cudaSuccess) {
      // the row padding beyond the halo is copied by the last tile of a row
      // but read by no MMA: zero it once
      cudaError_t ez = cudaMemset(c->xs, 0, lbrr::feature_source_bytes(c->g));
      if (ez == cudaSuccess) ez = lbrr::make_feature_map(c->xs, c->g, &c->xs_map);
      if (ez != cudaSuccess) {
        cudaGetLastError();
        cudaFree(c->xs);
        c->xs = nullptr;
        return fail(c, LB_ECUDA, "cannot prepare the feature source or its tensor map");
      }
    }
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, LB_ENOMEM, "cannot allocate the closure fields");
  }
  return LB_OK;
}

static int closure_capable(lb_ctx *c) {
  if (c->lattice != LB_D3Q27 || c->storage != LB_STORE_F32 || c->collision != LB_COLLIDE_RR ||
      c->g.walls)
    return fail(c, LB_EINVAL, "the learned closure needs a periodic D3Q27, FP32, RR context");
  return LB_OK;
}

int lb_closure_features(lb_ctx *c, const lb_mlp *m, void *X) {
  LB_CHECK_CTX(c);
  if (!m || !X) return fail(c, LB_EINVAL, "null argument");
  LB_NEED_DEVICE(c, X);
  int rc = closure_capable(c);
  if (rc == LB_OK) rc = ensure_mom(c, false);
  if (rc != LB_OK) return rc;
  DeviceGuard dg(c->device);
  cudaError_t e = lbrr::launch_moment_field(c->storage, c->f, c->g, c->parity, c->mom, c->stream);
  if (e == cudaSuccess) e = lbrr::launch_features(m->d, c->mom, c->g, X, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "closure features");
  return LB_OK;
}

int lb_closure_targets(lb_ctx *c, const lb_mlp *m, float *T) {
  LB_CHECK_CTX(c);
  if (!m || !T) return fail(c, LB_EINVAL, "null argument");
  LB_NEED_DEVICE(c, T);
  int rc = closure_capable(c);
  if (rc != LB_OK) return rc;
  DeviceGuard dg(c->device);
  cudaError_t e = lbrr::launch_targets(m->d, c->storage, c->f, c->g, c->parity, T, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "closure targets");
  return LB_OK;
}

static int coarsen(lb_ctx *fine, lb_ctx *coarse, double neq_scale) {
  LB_CHECK_CTX(fine);
  LB_CHECK_CTX(coarse);
  if (!std::isfinite(neq_scale)) return fail(coarse, LB_EINVAL, "neq_scale must be finite");
  if (fine->lattice != LB_D3Q27 || coarse->lattice != LB_D3Q27 || fine->storage != LB_STORE_F32 ||
      coarse->storage != LB_STORE_F32 || fine->g.walls || coarse->g.walls)
    return fail(coarse, LB_EINVAL, "coarsening needs two periodic D3Q27 FP32 contexts");
  if (fine->g.nx != 2 * coarse->g.nx || fine->g.ny != 2 * coarse->g.ny ||
      fine->g.nz != 2 * coarse->g.nz)
    return fail(coarse, LB_EINVAL, "the fine grid must be twice the coarse grid in every direction");
  if (fine->device != coarse->device) return fail(coarse, LB_EINVAL, "contexts on different devices");
  DeviceGuard dg(coarse->device);
  cudaError_t e = cudaSuccess;
  if (fine->stream != coarse->stream) e = cudaStreamSynchronize(fine->stream);
  if (e == cudaSuccess)
    e = lbrr::launch_coarsen(fine->storage, fine->f, fine->g, fine->parity, coarse->storage,
                             coarse->f, coarse->g, coarse->stream, (float)neq_scale);
  if (e != cudaSuccess) return cuda_fail(coarse, e, "coarsen");
  coarse->parity = 0;
  coarse->steps = 0;
  return LB_OK;
}

int lb_coarsen(lb_ctx *fine, lb_ctx *coarse) {
  Range nvtx_range("lb_coarsen");
  return coarsen(fine, coarse, 1.0);
}

int lb_coarsen_neq(lb_ctx *fine, lb_ctx *coarse, double neq_scale) {
  Range nvtx_range("lb_coarsen_neq");
  return coarsen(fine, coarse, neq_scale);
}

int lb_closure_step_targets(lb_ctx *pre, lb_ctx *post, const lb_mlp *m, float *T) {
  LB_CHECK_CTX(pre);
  LB_CHECK_CTX(post);
  if (!m || !T) return fail(pre, LB_EINVAL, "null argument");
  LB_NEED_DEVICE(pre, T);
  int rc = closure_capable(pre);
  if (rc == LB_OK) rc = closure_capable(post);
  if (rc != LB_OK) return rc;
  if (pre->g.nx != post->g.nx || pre->g.ny != post->g.ny || pre->g.nz != post->g.nz ||
      pre->device != post->device)
    return fail(pre, LB_EINVAL, "the two states must share the grid and the device");
  DeviceGuard dg(pre->device);
  cudaError_t e = cudaSuccess;
  if (post->stream != pre->stream) e = cudaStreamSynchronize(post->stream);
  if (e == cudaSuccess)
    e = lbrr::launch_step_targets(m->d, static_cast<const float *>(pre->f), pre->parity,
                                  static_cast<const float *>(post->f), post->parity, pre->g,
                                  (float)(1.0 - 1.0 / pre->tau), T, pre->stream);
  if (e != cudaSuccess) return cuda_fail(pre, e, "closure step targets");
  return LB_OK;
}

int lb_set_closure_ex(lb_ctx *c, const lb_mlp *m, float bound, float dead_zone) {
  LB_CHECK_CTX(c);
  if (!m) {
    c->closure = nullptr;
    return LB_OK;
  }
  if (!(bound > 0.f)) return fail(c, LB_EINVAL, "bound must be positive");
  if (!(dead_zone >= 0.f) || !std::isfinite(dead_zone))
    return fail(c, LB_EINVAL, "dead_zone must be a finite number >= 0");
  int rc = closure_capable(c);
  if (rc == LB_OK) rc = ensure_mom(c, true);
  if (rc != LB_OK) return rc;
  DeviceGuard dg(c->device);
  if (!c->fallbacks) {
    cudaError_t e = cudaMalloc(&c->fallbacks, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(c->fallbacks, 0, sizeof(unsigned long long));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(c, LB_ENOMEM, "cannot allocate the fallback counter");
    }
  }
  c->closure = m;
  c->closure_bound = bound;
  c->closure_dead_zone = dead_zone;
  return LB_OK;
}

int lb_set_closure(lb_ctx *c, const lb_mlp *m, float bound) {
  return lb_set_closure_ex(c, m, bound, 0.f);
}

int lb_closure_step_trace(lb_ctx *c, float *trace, void *xs_out) {
  LB_CHECK_CTX(c);
  if (!trace || !xs_out) return fail(c, LB_EINVAL, "null trace or feature-source buffer");
  LB_NEED_DEVICE(c, trace);
  LB_NEED_DEVICE(c, xs_out);
  if (!c->closure || !c->xs)
    return fail(c, LB_EINVAL,
                "needs a learned closure on a grid of whole 128-cell row tiles (lb_set_closure)");
  DeviceGuard dg(c->device);
  const float om1 = (float)(1.0 - 1.0 / c->tau);
  cudaError_t e = lbrr::launch_feature_source(c->closure->d, static_cast<const float *>(c->f),
                                              c->g, c->parity, c->xs, c->stream);
  if (e == cudaSuccess)
    e = lbrr::launch_mlp_conv_step(c->closure->d, c->xs_map, c->g, static_cast<float *>(c->f),
                                   om1, c->parity, c->fallbacks, c->closure_bound,
                                   c->closure_dead_zone, c->closure->status,
                                   c->closure->nblocks, c->stream, trace);
  if (e == cudaSuccess)
    e = lbrr::launch_export_features(c->xs, c->g, xs_out, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "closure step trace");
  c->parity ^= 1;
  ++c->steps;
  return LB_OK;
}

int lb_closure_fallbacks(lb_ctx *c, long long *count) {
  LB_CHECK_CTX(c);
  if (!count) return fail(c, LB_EINVAL, "null argument");
  *count = 0;
  if (!c->fallbacks) return LB_OK;
  DeviceGuard dg(c->device);
  unsigned long long h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, c->fallbacks, sizeof h, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "fallback counter");
  *count = (long long)h;
  if (c->closure) {
    int st = 0;
    e = cudaMemcpyAsync(&st, c->closure->status, sizeof st, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "closure status");
    if (st) {
      cudaMemsetAsync(c->closure->status, 0, sizeof(int), c->stream);
      return fail(c, LB_ETIMEOUT, "a tensor-core wait of the network timed out");
    }
  }
  return LB_OK;
}

// ---------------------------------------------------------- bounded waits

int lb_set_wait_limit(lb_ctx *c, int iterations) {
  LB_CHECK_CTX(c);
  if (iterations < 0) return fail(c, LB_EINVAL, "negative wait limit");
  DeviceGuard dg(c->device);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpy(c->status + 1, &iterations, sizeof(int), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(c, e, "set_wait_limit");
  return LB_OK;
}

int lb_mlp_set_wait_limit(lb_mlp *m, int iterations) {
  if (!m) return LB_EINVAL;
  if (iterations < 0) return mlp_fail(m, LB_EINVAL, "negative wait limit");
  DeviceGuard dg(m->device);
  cudaError_t e = cudaStreamSynchronize(m->stream);
  if (e == cudaSuccess)
    e = cudaMemcpy(m->status + 1, &iterations, sizeof(int), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return mlp_fail(m, LB_ECUDA, "set_wait_limit: %s", cudaGetErrorString(e));
  return LB_OK;
}

int lb_wait_selftest(int iterations) {
  if (iterations < 1) return lbrr::report_error(LB_EINVAL, "iterations must be >= 1");
  int *d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(d, 0, sizeof(int));
  if (e == cudaSuccess) e = lbrr::launch_wait_selftest((unsigned)iterations, d, nullptr);
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof h, cudaMemcpyDeviceToHost);
  if (d) cudaFree(d);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return lbrr::report_error(LB_ECUDA, "wait self-test: %s", cudaGetErrorString(e));
  }
  if (h != 1)
    return lbrr::report_error(LB_ECUDA, "a wait with no arrival completed (status %d)", h);
  return lbrr::report_error(LB_ETIMEOUT, "the bounded wait expired and was reported");
}

}  // extern "C"
