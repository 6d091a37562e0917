// Allocation-free variant of the CFL step-size reduction (perk_compute_dt_noalloc).
//
// Some callers must not allocate device memory at all: a solver embedded as a
// custom call inside another framework (an XLA/JAX custom call, a plugin of a
// larger simulation code) runs while that framework owns the device memory and
// its allocator, and a cudaMalloc there would bypass the framework's pool and
// implicitly synchronise the device. This entry point therefore takes its
// scratch space from a file-scope __device__ array that exists for as long as
// the library stays loaded, instead of from a context's buffers.

#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "perk.h"
#include "perk_internal.h"

namespace {

// Partial minima of the reduction (one per block) plus the final minimum.
// 8,193 doubles (64 KiB + 8 B) on every device that loads the library: enough for one block per
// DT_THREADS nodes of PERK_NOALLOC_MAX_ELEM cells, although the grid-stride reduction is launched
// with at most kLaunchBlocks blocks.
constexpr int kMaxBlocks = PERK_NOALLOC_MAX_ELEM / 16;
constexpr int kLaunchBlocks = 1024;
static_assert((int64_t)kMaxBlocks * perk::DT_THREADS >= (int64_t)PERK_NOALLOC_MAX_ELEM * perk::NODES,
              "scratch too small for one block per DT_THREADS nodes");
static_assert(kLaunchBlocks <= kMaxBlocks, "launch grid larger than the scratch");
static __device__ __align__(256) double g_dt_scratch[kMaxBlocks + 1];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_dt_scratch on the current device (the host-side symbol is
// only a stand-in).  Looked up once per device, with that device current.
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_dt_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" perk_status perk_compute_dt_noalloc(const double* d_U, const int32_t* d_level, int64_t n_elem,
                                               double length, double gamma, double cfl, void* stream, double* dt) {
  if (!d_U || !d_level || !dt || !(length > 0.0) || !(gamma > 1.0) || !(cfl > 0.0) || n_elem <= 0)
    return perk::set_context_free_error(PERK_E_INVALID_ARG, "perk_compute_dt_noalloc: invalid argument");
  if (n_elem > PERK_NOALLOC_MAX_ELEM)
    return perk::set_context_free_error(PERK_E_INVALID_ARG,
                                        "perk_compute_dt_noalloc: n_elem exceeds PERK_NOALLOC_MAX_ELEM (131072)");
  double* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess)
    return perk::set_context_free_error(PERK_E_CUDA, "perk_compute_dt_noalloc: cudaGetSymbolAddress failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t need = (n_elem * perk::NODES + perk::DT_THREADS - 1) / perk::DT_THREADS;
  const int n_blocks = (int)(need < kLaunchBlocks ? need : kLaunchBlocks);   // the reduction is grid-stride
  e = perk::launch_dt(st, n_elem, d_U, d_level, length, gamma, scratch, n_blocks, scratch + kMaxBlocks);
  if (e != cudaSuccess) return perk::set_context_free_error(PERK_E_CUDA, "perk_compute_dt_noalloc: launch failed");
  double m = 0.0;
  e = cudaMemcpyAsync(&m, scratch + kMaxBlocks, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess)
    return perk::set_context_free_error(PERK_E_CUDA, "perk_compute_dt_noalloc: reading the result failed");
  if (!std::isfinite(m) || !(m > 0.0))
    return perk::set_context_free_error(PERK_E_NONFINITE,
                                        "perk_compute_dt_noalloc: a node has no admissible wave speed");
  *dt = cfl * m / (double)perk::NN;
  return PERK_OK;
}
