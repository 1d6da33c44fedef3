// pdmcf_project.cu — the capped-simplex projection Pi (Zhang & Boyd, Sec. 2.3) as a
// standalone C ABI operation on device arrays (mcf_project_capped_simplex).
//
// The kernel is the edge phase's projection (warm-started Newton on
// phi(mu) = sum (q - mu)_+ - c with exact active-set finish) applied to caller-provided
// columns. Per-column FP64 squared distances go to scratch memory and are summed in a fixed
// order, so the reported distance does not depend on the launch grid.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "pdmcf_internal.h"
#include "pdmcf_kernels.h"

namespace pdmcf {

// Fixed-order sum of x[0..count) into *out by one block of 1024 threads.
__global__ void __launch_bounds__(1024) fixed_order_sum_kernel(const double* x, long long count,
                                                               double* out) {
  __shared__ double sh[1024];
  const long long per = (count + 1023) / 1024;
  const long long b0 = (long long)threadIdx.x * per;
  long long b1 = b0 + per;
  if (b1 > count) b1 = count;
  double s = 0.0;
  for (long long b = b0; b < b1; ++b) s += x[b];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int off = 512; off > 0; off >>= 1) {
    if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

using ProjKernel = void (*)(ProjArgs);

template <int IDX>
static void fill_proj(ProjKernel* t) {
  constexpr ShapeDesc d = kShapes[IDX];
  constexpr int MB = min_blocks<float, d.vpt, 4, d.block>();
  t[IDX] = project_kernel<d.vpt, d.group, d.block, MB>;
}

const ProjKernel* proj_table() {
  static ProjKernel t[NUM_SHAPES] = {};
  static bool init = [] {
    fill_proj<0>(t); fill_proj<1>(t); fill_proj<2>(t); fill_proj<3>(t); fill_proj<4>(t);
    fill_proj<5>(t); fill_proj<6>(t); fill_proj<7>(t); fill_proj<8>(t); fill_proj<9>(t);
    fill_proj<10>(t); fill_proj<11>(t); fill_proj<12>(t); fill_proj<13>(t);
    return true;
  }();
  (void)init;
  return t;
}

// Launches the projection and the fixed-order sum into scratch[m], and copies the sum to
// *dist2 (if not NULL). scratch must hold m + 1 doubles; arguments already validated.
int project_launch(int32_t n, int32_t m, int32_t ld, const float* Qt, const float* cap,
                   float* Ft, float* mu, double* dist2, cudaStream_t st, double* scratch) {
  const int nchunks = ld / 4;
  const int shape = pick_shape(nchunks);
  const ShapeDesc sd = kShapes[shape];
  const ProjKernel fn = proj_table()[shape];
  int dev = 0, sms = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)fn, sd.block, 0);
  if (e != cudaSuccess) {
    set_error(std::string("CUDA error ") + cudaGetErrorString(e));
    return MCF_ERR_CUDA;
  }
  const int gpb = sd.block / sd.group;
  const int need = (m + gpb - 1) / gpb;
  const int grid = need < (occ > 0 ? occ : 1) * sms ? need : (occ > 0 ? occ : 1) * sms;
  ProjArgs a{n, m, ld, Qt, cap, Ft, mu, scratch};
  void* kargs[] = {&a};
  e = cudaLaunchKernel((const void*)fn, dim3(grid > 0 ? grid : 1), dim3(sd.block), kargs, 0, st);
  if (e == cudaSuccess) {
    fixed_order_sum_kernel<<<1, 1024, 0, st>>>(scratch, (long long)m, scratch + m);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && dist2) {
    e = cudaMemcpyAsync(dist2, scratch + m, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) {
    set_error(std::string("CUDA error ") + cudaGetErrorString(e));
    return MCF_ERR_CUDA;
  }
  return MCF_OK;
}

int project_validate(int32_t n, int32_t m, int32_t ld, const float* Qt, const float* cap,
                     const float* Ft, const float* mu) {
  if (n < 1 || m < 0 || ld < n || (ld % 4) != 0) {
    set_error("need n >= 1, m >= 0, ld >= n and ld a multiple of 4");
    return MCF_ERR_INVALID;
  }
  if (m > 0 && (!Qt || !cap || !Ft || !mu)) {
    set_error("Qt, cap, Ft and mu must be device pointers");
    return MCF_ERR_INVALID;
  }
  if (((uintptr_t)Qt | (uintptr_t)Ft) % 16 != 0) {
    set_error("Qt and Ft must be 16-byte aligned");
    return MCF_ERR_INVALID;
  }
  if (pick_shape(ld / 4) < 0) {
    set_error("ld too large (at most 32768 floats per column)");
    return MCF_ERR_INVALID;
  }
  return MCF_OK;
}

}  // namespace pdmcf

using namespace pdmcf;

extern "C" int mcf_project_capped_simplex(int32_t n, int32_t m, int32_t ld, const float* Qt,
                                          const float* cap, float* Ft, float* mu,
                                          double* dist2, void* stream) {
  int rc = project_validate(n, m, ld, Qt, cap, Ft, mu);
  if (rc != MCF_OK) return rc;
  if (m == 0) {
    if (dist2) *dist2 = 0.0;
    return MCF_OK;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double* scratch = nullptr;
  if (cudaMalloc((void**)&scratch, ((size_t)m + 1) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation of the projection scratch failed");
    return MCF_ERR_OOM;
  }
  rc = project_launch(n, m, ld, Qt, cap, Ft, mu, dist2, st, scratch);
  cudaError_t e = cudaStreamSynchronize(st);   // the scratch must outlive the kernels
  cudaFree(scratch);
  if (rc == MCF_OK && e != cudaSuccess) {
    set_error(std::string("CUDA error ") + cudaGetErrorString(e));
    rc = MCF_ERR_CUDA;
  }
  return rc;
}
