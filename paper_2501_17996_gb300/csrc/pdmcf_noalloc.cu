// pdmcf_noalloc.cu — mcf_project_capped_simplex_noalloc: the projection entry point for
// callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc (or let a library call it for them): code that runs
// while a CUDA graph is being captured, processes whose device memory is handed out by their
// own pool or by a framework allocator, and real-time loops that must not enter the
// allocator. This variant runs the same projection kernel as mcf_project_capped_simplex, but
// its scratch (one double per column plus one for the total) lives in the fixed array below,
// which every GPU that loads this library holds until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "pdmcf_internal.h"

namespace pdmcf {
int project_validate(int32_t n, int32_t m, int32_t ld, const float* Qt, const float* cap,
                     const float* Ft, const float* mu);
int project_launch(int32_t n, int32_t m, int32_t ld, const float* Qt, const float* cap,
                   float* Ft, float* mu, double* dist2, cudaStream_t st, double* scratch);
}  // namespace pdmcf

// Largest column count the fixed scratch serves: 262144 columns, 2 MiB of doubles.
#define MCF_NOALLOC_MAX_COLS (1 << 18)

// Per-column squared distances [0, m) and their fixed-order total [m]. Each call writes
// every entry it reads, so nothing has to be cleared between calls.
static __device__ __align__(256) double g_noalloc_scratch[MCF_NOALLOC_MAX_COLS + 1];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device
// (with that device current). In host code the array's name is only a host-side stand-in,
// so kernels must be given this address instead.
int scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    pdmcf::set_error(std::string("CUDA error ") + cudaGetErrorString(e));
    return MCF_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    pdmcf::set_error("device ordinal out of range for the no-alloc scratch table");
    return MCF_ERR_INVALID;
  }
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_scratch_addr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      pdmcf::set_error(std::string("cudaGetSymbolAddress of the no-alloc scratch failed: ") +
                       cudaGetErrorString(e));
      return MCF_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return MCF_OK;
}
}  // namespace

extern "C" int mcf_project_capped_simplex_noalloc(int32_t n, int32_t m, int32_t ld,
                                                  const float* Qt, const float* cap, float* Ft,
                                                  float* mu, double* dist2, void* stream) {
  int rc = pdmcf::project_validate(n, m, ld, Qt, cap, Ft, mu);
  if (rc != MCF_OK) return rc;
  if (m > MCF_NOALLOC_MAX_COLS) {
    pdmcf::set_error("m exceeds the no-alloc maximum of 262144 columns; use "
                     "mcf_project_capped_simplex");
    return MCF_ERR_INVALID;
  }
  if (m == 0) {
    if (dist2) *dist2 = 0.0;
    return MCF_OK;
  }
  double* scratch = nullptr;
  rc = scratch_address(&scratch);
  if (rc != MCF_OK) return rc;
  return pdmcf::project_launch(n, m, ld, Qt, cap, Ft, mu, dist2, (cudaStream_t)stream, scratch);
}
