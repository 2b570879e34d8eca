// lb_diagnostics_static: the mass / momentum / kinetic-energy reduction of
// lb_diagnostics for callers that cannot allocate device memory.
//
// Who needs it: a caller that holds a population store in memory it manages
// itself (a checkpoint copy from lb_get_state, or a buffer carved from its
// own allocator) and that may not call cudaMalloc/cudaFree: its device memory
// is already fully reserved by another allocator, or it runs beside a live
// simulation and must not take the device-wide synchronisation that
// cudaFree implies. It brings the input and the output; the partial sums of
// the reduction live in a fixed, file-scope device array instead of memory
// allocated per call or per context.
//
// The array holds one row of partial sums per block of kCellsPerBlock cells
// plus the result row, sized for LB_STATIC_MAX_CELLS cells (1.25 MiB). Every
// GPU that loads the library holds it until the process exits. All calls on
// a device share it: calls that overlap on the GPU (different streams, or
// different host threads) race on it and must be serialised by the caller.
// Every row a call reads is written earlier in the same call, so nothing has
// to be cleared between calls.
//
// The device address of the array is looked up once per device and CUDA
// context, on the first call made while that context is current
// (cudaGetSymbolAddress); a new context on the device (after cudaDeviceReset,
// or a context the caller created itself) is looked up again on its first
// call. Make that first call before any stream capture on the device.
//
// The store must be device (or managed) memory of the current device: a host
// pointer, or memory of another GPU, is rejected with LB_EINVAL before any
// kernel could touch it (cudaPointerGetAttributes, which allocates nothing).
#include <cuda.h>

#include <cstring>
#include <mutex>

#include "lbrr.h"
#include "lbrr_launch.h"

namespace {

constexpr long long kCellsPerBlock = 4096;  // 16 cells per thread
constexpr int kRows = (int)(LB_STATIC_MAX_CELLS / kCellsPerBlock);
static_assert(LB_STATIC_MAX_CELLS % kCellsPerBlock == 0, "whole rows");

// kRows partial rows, then the result row
static __device__ __align__(256) double g_scratch[(kRows + 1) * lbrr::kRedValues];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct ScratchSlot {
  CUcontext ctx;  // the context the address was looked up in
  double *addr;
};
ScratchSlot g_slot[kMaxDevices] = {};

// The driver's cuCtxGetCurrent, found through the runtime (no link to libcuda).
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<CtxGetCurrentFn>(p);
  }();
  return fn;
}

// Device address of g_scratch in the current context of the current device
// (looked up once per device and context).
int scratch_address(int dev, double **out) {
  if (dev < 0 || dev >= kMaxDevices)
    return lbrr::report_error(LB_EINVAL, "lb_diagnostics_static: device %d out of range", dev);
  CtxGetCurrentFn get = ctx_get_current();
  CUcontext ctx = nullptr;
  if (!get || get(&ctx) != CUDA_SUCCESS || !ctx)
    return lbrr::report_error(LB_ECUDA, "lb_diagnostics_static: no current CUDA context");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_slot[dev].addr || g_slot[dev].ctx != ctx) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
      return lbrr::report_error(LB_ECUDA,
                                "lb_diagnostics_static: cudaGetSymbolAddress failed (%s)",
                                cudaGetErrorString(e));
    g_slot[dev] = ScratchSlot{ctx, static_cast<double *>(p)};
  }
  *out = g_slot[dev].addr;
  return LB_OK;
}

// LB_OK when `store` is device or managed memory that the current device
// `dev` can read as its own.
int check_store(const void *store, int dev) {
  cudaPointerAttributes a{};
  cudaError_t e = cudaPointerGetAttributes(&a, store);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return lbrr::report_error(LB_EINVAL, "lb_diagnostics_static: the store is not CUDA memory (%s)",
                              cudaGetErrorString(e));
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
    return lbrr::report_error(LB_EINVAL,
                              "lb_diagnostics_static: the store must be device memory of the "
                              "current device (got a host or unregistered pointer)");
  if (a.type == cudaMemoryTypeDevice && a.device != dev)
    return lbrr::report_error(LB_EINVAL,
                              "lb_diagnostics_static: the store lives on device %d, the current "
                              "device is %d",
                              a.device, dev);
  return LB_OK;
}

}  // namespace

extern "C" int lb_diagnostics_static(int lattice, int nx, int ny, int nz, int storage, int parity,
                                     const void *store, double *out, void *stream) {
  if (!store || !out) return lbrr::report_error(LB_EINVAL, "lb_diagnostics_static: null pointer");
  if (lattice != LB_D2Q9 && lattice != LB_D3Q19 && lattice != LB_D3Q27)
    return lbrr::report_error(LB_EINVAL, "lb_diagnostics_static: unknown lattice %d", lattice);
  if (nx < 1 || ny < 1 || nz < 1 || (lattice == LB_D2Q9 && nz != 1))
    return lbrr::report_error(LB_EINVAL, "lb_diagnostics_static: bad grid %d x %d x %d", nx, ny,
                              nz);
  if (storage < LB_STORE_F32 || storage > LB_STORE_BF16)
    return lbrr::report_error(LB_EINVAL, "lb_diagnostics_static: unknown storage %d", storage);
  if (parity != 0 && parity != 1)
    return lbrr::report_error(LB_EINVAL, "lb_diagnostics_static: parity must be 0 or 1");
  const long long n = (long long)nx * ny * nz;
  if (n > LB_STATIC_MAX_CELLS)
    return lbrr::report_error(LB_EINVAL,
                              "lb_diagnostics_static: %lld cells exceed the static scratch limit "
                              "of %lld cells (LB_STATIC_MAX_CELLS); use lb_diagnostics",
                              n, (long long)LB_STATIC_MAX_CELLS);
  int dev = -1;
  cudaError_t de = cudaGetDevice(&dev);
  if (de != cudaSuccess)
    return lbrr::report_error(LB_ECUDA, "lb_diagnostics_static: no CUDA device (%s)",
                              cudaGetErrorString(de));
  int rc = check_store(store, dev);
  if (rc != LB_OK) return rc;
  double *scratch = nullptr;
  rc = scratch_address(dev, &scratch);
  if (rc != LB_OK) return rc;
  const int nblocks = (int)((n + kCellsPerBlock - 1) / kCellsPerBlock);
  double *result = scratch + (long long)kRows * lbrr::kRedValues;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const lbrr::Grid g{nx, ny, nz, n};
  cudaError_t e = lbrr::launch_diagnostics_blocks(lattice, storage, store, g, parity, nblocks,
                                                  scratch, result, st);
  double h[lbrr::kRedValues];
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, result, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess)
    return lbrr::report_error(LB_ECUDA, "lb_diagnostics_static: %s", cudaGetErrorString(e));
  const int d = lattice == LB_D2Q9 ? 2 : 3;
  out[0] = (double)n + h[0];
  for (int a = 0; a < d; ++a) out[1 + a] = h[1 + a];
  out[1 + d] = h[4];
  for (int k = 0; k < 2 + d; ++k)
    if (!(out[k] - out[k] == 0.0))
      return lbrr::report_error(LB_EDIVERGED, "lb_diagnostics_static: diagnostic %d is not finite",
                                k);
  return LB_OK;
}
