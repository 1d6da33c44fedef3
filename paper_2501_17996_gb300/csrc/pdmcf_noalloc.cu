// pdmcf_noalloc.cu — mcf_project_capped_simplex_noalloc: the projection entry point for
// callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc (or let a library call it for them): processes whose
// device memory is handed out by their own pool or by a framework allocator that must see
// every allocation, and real-time loops that must not enter the allocator (a cudaMalloc can
// synchronize the device and take milliseconds). This variant runs the same projection
// kernel as mcf_project_capped_simplex, but its scratch (one double per column plus one for
// the total) lives in the fixed array below, which every GPU that loads this library holds
// until the process exits.
#include <cuda.h>   // CUcontext and CUresult only: the two driver calls come through cudart
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

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Unique id of the calling thread's current context (0 if none or not available). The
// driver functions are reached through cudart, so the library needs no link to libcuda.
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(fn);
    fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(fn);
  });
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}
}  // namespace pdmcf

// Largest column count the fixed scratch serves: 262144 columns, 2 MiB of doubles.
#define MCF_NOALLOC_MAX_COLS (1 << 18)

// Per-column squared distances [0, m) and their fixed-order total [m]. Each call writes
// every entry it reads, so nothing has to be cleared between calls.
static __device__ __align__(256) double g_noalloc_scratch[MCF_NOALLOC_MAX_COLS + 1];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct ScratchAddr {
  unsigned long long ctx_id = 0;   // context the address belongs to (0: not looked up)
  double* addr = nullptr;
};
ScratchAddr g_scratch[kMaxDevices];

// Device address of the scratch array in the current device's context. In host code the
// array's name is only a host-side stand-in, so kernels must be given this address. It is
// looked up with the device current on the first call per device, and again whenever the
// context has changed since (a cudaDeviceReset by the application destroys the context that
// held the old address).
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
  ScratchAddr& s = g_scratch[dev];
  const unsigned long long ctx = pdmcf::current_context_id();
  if (!s.addr || ctx == 0 || ctx != s.ctx_id) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      pdmcf::set_error(std::string("cudaGetSymbolAddress of the no-alloc scratch failed: ") +
                       cudaGetErrorString(e));
      return MCF_ERR_CUDA;
    }
    s.addr = p;
    s.ctx_id = pdmcf::current_context_id();   // the lookup makes the primary context current
  }
  *out = s.addr;
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
