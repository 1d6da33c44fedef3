// pdmcf_solver.cu — host driver of the PDMCF iteration on one GPU.
//
// Owns the device state of a problem (iterates, incidence, data, reduction scratch),
// launches one iteration as edge -> node -> [check] -> scalar kernels, groups k_check
// iterations into a CUDA graph whose last iteration evaluates the stop test quantities,
// and reads the FP64 scalars back once per chunk (Algorithm 2.1, step 1, evaluated every
// k_check iterations).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <type_traits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "pdmcf_batch.cuh"
#include "pdmcf_internal.h"
#include "pdmcf_kernels.h"

namespace pdmcf {

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      set_error(std::string("CUDA error ") + cudaGetErrorString(e_) + " in " #call);   \
      return MCF_ERR_CUDA;                                                             \
    }                                                                                  \
  } while (0)

// ------------------------------------------------------------------ scalar tail kernel

struct ScalarArgs {
  DevScalars* sc;
  const double* pe;
  int nbe;
  const double* pn;
  int nbn;
  const double* pc;
  int nbc;
  int check;
};

__global__ void __launch_bounds__(256) scalar_kernel(ScalarArgs a) {
  __shared__ double sh[256];
  const double dF2 = det_sum(a.pe, a.nbe, 1, 0, sh);
  const double dY2 = det_sum(a.pn, a.nbn, NODE_PARTS, 0, sh);
  double nodep[NODE_PARTS];
  double chk[CHECK_PARTS];
  if (a.check) {
    for (int f = 1; f < NODE_PARTS; ++f) nodep[f] = det_sum(a.pn, a.nbn, NODE_PARTS, f, sh);
    for (int f = 0; f < CHECK_PARTS; ++f) chk[f] = det_sum(a.pc, a.nbc, CHECK_PARTS, f, sh);
  }
  if (threadIdx.x != 0) return;
  scalar_update(a.sc, dF2, dY2, nodep, chk, a.check != 0);
}

// ------------------------------------------------------------------ init / output kernels

// Y^0 = I - 1 1^T (Sec. 2.5): 0 on the diagonal, -1 elsewhere; pads 0.
template <typename P>
__global__ void init_y_kernel(P* Y, int n, int ld) {
  const size_t total = (size_t)n * ld;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx / ld), i = (int)(idx % ld);
    Y[idx] = (i < n && i != j) ? P(-1) : P(0);
  }
}

// F^ = (q - mu)_+ with q = F^{k-3/2} + alpha_last (Y^{k-1}_{:,h} - Y^{k-1}_{:,t}): the
// projected flow the last iteration computed (Algorithm 2.1 returns F^{k-1/2}), formed in the
// frame shifted by that iteration's multiplier (hi/lo pair) as the edge phase formed it.
template <typename P, typename S>
__global__ void fhat_kernel(const S* Fo, const P* Y, const __nv_bfloat16* Ylo, const int32_t* et,
                            const int32_t* eh, const P* mu, const P* mu_lo, const DevScalars* sc,
                            P* out, int m, int ld) {
  const P alpha = (P)sc->alpha_last;
  const size_t total = (size_t)m * ld;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int e = (int)(idx / ld), i = (int)(idx % ld);
    const size_t ih = (size_t)eh[e] * ld + i, it = (size_t)et[e] * ld + i;
    P dl = P(0);
    if (Ylo) dl = (P)(__bfloat162float(Ylo[ih]) - __bfloat162float(Ylo[it]));
    const P q = shifted_q<P>(to_p<P>(Fo[idx]), Y[ih], Y[it], dl, alpha, mu[e], mu_lo[e]);
    out[idx] = q > P(0) ? q : P(0);
  }
}

// ------------------------------------------------------------------ device state

// NVTX ranges (host side) for profilers: a solve, each chunk of k_check iterations and, in
// timed solves, each phase's launch. Without an attached tool they cost a branch.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

struct DeviceState {
  int device = -1, precision = -1;
  int n = 0, m = 0, ld = 0;
  size_t sbytes = 0, pbytes = 0;
  void* F[2] = {nullptr, nullptr};
  void* Y[2] = {nullptr, nullptr};
  void* Ylo[2] = {nullptr, nullptr};   // compensated-dual tails (FP32/BF16 iterates)
  bool lo_live = false;                 // the tails match the resident Y
  void *Pm = nullptr, *W = nullptr, *G = nullptr, *mu = nullptr, *cap = nullptr;
  void *That = nullptr, *Uprime = nullptr, *Yhat = nullptr;
  int32_t *e_tail = nullptr, *e_head = nullptr, *in_ptr = nullptr, *out_ptr = nullptr,
          *out_idx = nullptr;
  double *part_edge = nullptr, *part_node = nullptr, *part_check = nullptr;
  DevScalars* sc = nullptr;
  DevScalars* sc_host = nullptr;
  cudaStream_t own_stream = nullptr;
  cudaMemPool_t pool = nullptr;   // where the buffers below come from (nullptr: cudaMalloc)
  int shape = -1, auto_shape = -1, block = 0, grid_edge = 0, grid_node = 0, grid_check = 0;
  int requested_shape = -1;   // mcf_options.shape the grids were configured for
  // pipelined edge phase (tma >= 0): one CTA per SM over head-aligned edge ranges
  int tma = -1, tma_kind = 0, grid_tma = 0, grid_node_pin = 0;   // kind 1 bulk-copy, 2 in-sum
  bool renumbered = false;   // nodes relabelled for locality (Topology::node_of)
  size_t tma_smem = 0;
  void* Pin = nullptr;
  int32_t* cta_ptr = nullptr;
  int32_t* node_map = nullptr;   // caller node -> internal node (boundary layouts)
  int cur = 0;
  bool valid = false;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int graph_len = 0;
  double graph_rho = 0.0;
  cudaStream_t graph_stream = nullptr;
  bool graph_lo = false;
  bool graphs_broken = false;
};

template <typename P, typename S> const KernelTable<P, S>& get_table();
template <> const KernelTable<float, float>& get_table<float, float>() {
  static const KernelTable<float, float> t = [] {
    KernelTable<float, float> t{};
    fill_f32_0(t); fill_f32_1(t); fill_f32_2(t); fill_f32_3(t); fill_f32_4(t);
    return t;
  }();
  return t;
}
template <> const KernelTable<double, double>& get_table<double, double>() {
  static const KernelTable<double, double> t = [] {
    KernelTable<double, double> t{};
    fill_f64_0(t); fill_f64_1(t); fill_f64_2(t); fill_f64_3(t); fill_f64_4(t);
    return t;
  }();
  return t;
}
template <> const KernelTable<float, __nv_bfloat16>& get_table<float, __nv_bfloat16>() {
  static const KernelTable<float, __nv_bfloat16> t = [] {
    KernelTable<float, __nv_bfloat16> t{};
    fill_bf16_0(t); fill_bf16_1(t); fill_bf16_2(t); fill_bf16_3(t); fill_bf16_4(t);
    return t;
  }();
  return t;
}

static void destroy_graphs(DeviceState* d) {
  for (int i = 0; i < 2; ++i)
    if (d->graph[i]) { cudaGraphExecDestroy(d->graph[i]); d->graph[i] = nullptr; }
  d->graph_len = 0;
}

// ------------------------------------------------------------------ device memory
// A problem's device state (about 11 GB at n = 10^4, m = 10^5) and the boundary's staging
// buffers come from one stream-ordered memory pool per device, which keeps up to 32 GB of
// freed memory for reuse: releasing a state with cudaFree took 12 ms at that size, and every
// cold solve of a new network paid it and the allocations again. The pool is created again
// when the device's context has changed (a cudaDeviceReset by the application); a device
// without memory pools uses cudaMalloc/cudaFree.
namespace {
struct PoolSlot {
  cudaMemPool_t pool = nullptr;
  unsigned long long ctx = 0;
  bool unsupported = false;
};
constexpr int kPoolDevices = 64;
std::mutex g_pool_mu;
PoolSlot g_pools[kPoolDevices];
}  // namespace

static cudaMemPool_t state_pool(int device) {
  if (device < 0 || device >= kPoolDevices) return nullptr;
  std::lock_guard<std::mutex> g(g_pool_mu);
  PoolSlot& s = g_pools[device];
  if (s.unsupported) return nullptr;
  const unsigned long long ctx = current_context_id();
  if (s.pool && (ctx == 0 || ctx == s.ctx)) return s.pool;
  int ok = 0;
  if (cudaDeviceGetAttribute(&ok, cudaDevAttrMemoryPoolsSupported, device) != cudaSuccess || !ok) {
    cudaGetLastError();
    s.unsupported = true;
    return nullptr;
  }
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
    cudaGetLastError();
    s.unsupported = true;
    return nullptr;
  }
  uint64_t keep = (uint64_t)32 << 30;
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  s.pool = pool;
  s.ctx = ctx;
  return pool;
}

// The kernels' vector loads and bulk copies need 16-byte aligned buffers (cudaMalloc returns
// 256-byte aligned ones); a buffer that is not aligned is refused rather than used.
static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Frees a state buffer; the caller has made sure no device work still uses it (as cudaFree
// does by synchronizing the device).
static void dfree(DeviceState* d, void* p) {
  if (!p) return;
  if (d->pool) cudaFreeAsync(p, d->own_stream);
  else cudaFree(p);
}

// A buffer of the state, ready for use on any stream when this returns.
static bool dalloc(DeviceState* d, void** p, size_t bytes) {
  *p = nullptr;
  cudaError_t e;
  if (d->pool) {
    e = cudaMallocFromPoolAsync(p, bytes, d->pool, d->own_stream);
    if (e == cudaErrorMemoryAllocation) {   // return the pool's cached memory and retry
      cudaGetLastError();
      cudaStreamSynchronize(d->own_stream);
      cudaMemPoolTrimTo(d->pool, 0);
      e = cudaMallocFromPoolAsync(p, bytes, d->pool, d->own_stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->own_stream);
  } else {
    e = cudaMalloc(p, bytes);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  if (!aligned16(*p)) {
    dfree(d, *p);
    *p = nullptr;
    return false;
  }
  return true;
}

// A staging buffer used on stream st only: allocated, used and freed in st's order.
static void sfree(DeviceState* d, void* p, cudaStream_t st) {
  if (!p) return;
  if (d->pool) cudaFreeAsync(p, st);
  else cudaFree(p);
}
static bool salloc(DeviceState* d, void** p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  const cudaError_t e = d->pool ? cudaMallocFromPoolAsync(p, bytes, d->pool, st) : cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  if (!aligned16(*p)) {
    sfree(d, *p, st);
    *p = nullptr;
    return false;
  }
  return true;
}

static void free_state(DeviceState* d) {
  if (!d) return;
  cudaSetDevice(d->device);
  destroy_graphs(d);
  cudaDeviceSynchronize();   // no kernel or copy may still use the buffers
  void* bufs[] = {d->F[0], d->F[1], d->Y[0], d->Y[1], d->Ylo[0], d->Ylo[1], d->Pm, d->W, d->G, d->mu, d->cap,
                  d->That, d->Uprime, d->Yhat, d->e_tail, d->e_head, d->in_ptr,
                  d->out_ptr, d->out_idx, d->part_edge, d->part_node, d->part_check, d->sc,
                  d->Pin, d->cta_ptr, d->node_map};
  for (void* b : bufs) dfree(d, b);
  if (d->sc_host) cudaFreeHost(d->sc_host);
  if (d->own_stream) cudaStreamDestroy(d->own_stream);
  delete d;
}

static size_t ld_of(int n) { return (size_t)((n + 7) / 8 * 8); }

static size_t elem_bytes_f(int precision) {
  return precision == MCF_FP64 ? 8 : (precision == MCF_BF16_F ? 2 : 4);
}
static size_t elem_bytes_p(int precision) { return precision == MCF_FP64 ? 8 : 4; }

int64_t device_bytes(const mcf_problem* p, int precision) {
  const size_t ld = ld_of(p->n), n = p->n, m = p->m;
  const size_t sf = elem_bytes_f(precision), sp = elem_bytes_p(precision);
  size_t b = 2 * m * ld * sf;                       // F ping-pong
  b += 2 * n * ld * sp;                             // Y ping-pong
  if (precision != MCF_FP64) b += 2 * n * ld * 2;   // compensated-dual tails
  b += (3 + (p->gamma_mat.empty() ? 0 : 1)) * n * ld * sp;   // P, W, [gamma], T^ (+below)
  b += 2 * n * ld * sp;                             // U', Y^
  b += 3 * m * sp + (3 * m + 2 * (n + 1)) * 4;      // mu (hi/lo), cap, incidence
  b += 64 * 1024;                                   // partials, scalars
  return (int64_t)b;
}

// Upload c, w (transposed to Wt[j][i] = w_ij) and per-pair gamma in precision P.
// ------------------------------------------------------------------ boundary layouts
// The caller's arrays are row-major n x n (or n x m for F) in doubles; the device keeps
// source-major rows in its own node numbering. Both conversions run on the device as tiled
// transposes (32 x 32 tiles through shared memory, so reads and writes are coalesced), over
// chunks of rows so the staging buffer stays small.

// out[r][c] (r in [r0, r0 + rows), c < ncols, doubles) = in[rowmap[c]][colmap[r]]
template <typename P>
__global__ void gather_out_kernel(const P* __restrict__ in, size_t ld_in,
                                  const int32_t* __restrict__ rowmap,
                                  const int32_t* __restrict__ colmap, double* __restrict__ out,
                                  int r0, int rows, int ncols) {
  __shared__ double tile[32][33];
  const int rb = blockIdx.y * 32, cb = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int k = ty; k < 32; k += 8) {          // read: consecutive threads -> consecutive r
    const int r = rb + tx, c = cb + k;
    if (r < rows && c < ncols)
      tile[k][tx] = (double)in[(size_t)rowmap[c] * ld_in + colmap[r0 + r]];
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {          // write: consecutive threads -> consecutive c
    const int r = rb + k, c = cb + tx;
    if (r < rows && c < ncols) out[(size_t)r * ncols + c] = tile[tx][k];
  }
}

// W[node(c)][node(r0 + r)] = in[r][c] for the chunk's caller rows r (diag: `diag`)
template <typename P>
__global__ void scatter_in_kernel(const double* __restrict__ in, int r0, int rows, int n,
                                  const int32_t* __restrict__ node, P* __restrict__ W,
                                  size_t ld, P diag) {
  __shared__ double tile[32][33];
  const int rb = blockIdx.y * 32, cb = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int k = ty; k < 32; k += 8) {          // read along c
    const int r = rb + k, c = cb + tx;
    if (r < rows && c < n) tile[k][tx] = in[(size_t)r * n + c];
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {          // write along r (the internal column)
    const int r = rb + tx, c = cb + k;
    if (r < rows && c < n) {
      const int i = r0 + r;
      W[(size_t)node[c] * ld + node[i]] = (i == c) ? diag : (P)tile[tx][k];
    }
  }
}

// Node map (caller node -> internal node) on the device, uploaded once per state.
static int ensure_node_map(mcf_problem* p, DeviceState* d, cudaStream_t st) {
  if (d->node_map) return MCF_OK;
  std::vector<int32_t> nm(d->n);
  for (int i = 0; i < d->n; ++i) nm[i] = p->topo.node(i);
  if (!dalloc(d, (void**)&d->node_map, (size_t)d->n * 4)) {
    set_error("device allocation failed");
    return MCF_ERR_OOM;
  }
  CK(cudaMemcpyAsync(d->node_map, nm.data(), (size_t)d->n * 4, cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  return MCF_OK;
}

// Rows of the caller's n x n array per staging chunk (about 64 MB of doubles).
static int chunk_rows(int n, int cols) {
  const size_t per = (size_t)cols * sizeof(double);
  return (int)std::max<size_t>(32, std::min<size_t>((size_t)n, ((size_t)64 << 20) / per));
}

// Upload c and w (placed as Wt[node(j)][node(i)] = w_ij) and per-pair gamma in precision P.
template <typename P>
static int upload_data(mcf_problem* p, DeviceState* d, cudaStream_t st) {
  const int n = p->n, m = p->m;
  const size_t ld = d->ld;
  std::vector<P> cap(m);
  for (int e = 0; e < m; ++e) cap[e] = (P)p->cap[p->topo.perm[e]];
  CK(cudaMemcpyAsync(d->cap, cap.data(), m * sizeof(P), cudaMemcpyHostToDevice, st));
  int rc = ensure_node_map(p, d, st);
  if (rc != MCF_OK) return rc;
  const int rows = chunk_rows(n, n);
  double* stage = nullptr;
  if (!salloc(d, (void**)&stage, (size_t)rows * n * sizeof(double), st)) {
    set_error("device allocation for the weight upload failed");
    return MCF_ERR_OOM;
  }
  auto place = [&](const double* src, void* dst, P diag) -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(dst, 0, (size_t)n * ld * sizeof(P), st);   // pads stay 0
    for (int r0 = 0; r0 < n && e == cudaSuccess; r0 += rows) {
      const int nr = std::min(rows, n - r0);
      e = cudaMemcpyAsync(stage, src + (size_t)r0 * n, (size_t)nr * n * sizeof(double),
                          cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) break;
      const dim3 grid((n + 31) / 32, (nr + 31) / 32);
      scatter_in_kernel<P><<<grid, dim3(32, 8), 0, st>>>(stage, r0, nr, n, d->node_map,
                                                         (P*)dst, ld, diag);
      e = cudaGetLastError();
    }
    return e;
  };
  cudaError_t e = place(p->w.data(), d->W, P(0));
  if (e == cudaSuccess && d->G) e = place(p->gamma_mat.data(), d->G, P(0.5));
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the stage and the host vectors
  sfree(d, stage, st);
  CK(e);
  p->data_dirty = false;
  return MCF_OK;
}

int mcf_shape_count() { return NUM_SHAPES + 2 * NUM_TMA; }

template <typename S> const TmaTable<S>& get_tma_table();
template <> const TmaTable<float>& get_tma_table<float>() { return tma_table_f32(); }
template <> const TmaTable<__nv_bfloat16>& get_tma_table<__nv_bfloat16>() { return tma_table_bf16(); }

// Pipelined path for shape index NUM_SHAPES + t (t < NUM_TMA); needs two stages of
// (F row + Y row) in shared memory.
template <typename S>
static int setup_tma(DeviceState* d, int want) {
  constexpr int VW = RowTraits<S>::VW;
  const int nchunks = (int)(d->ld / VW);
  int smem_optin = 0, sms = 0;
  CK(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, d->device));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d->device));
  // kind 1: bulk-copy pipeline, two stages of (F row + Y row), one CTA per SM
  // kind 2: register edge phase with in-sums, (Y row + in-sum row) per CTA, two CTAs per SM
  const size_t smem1 = 2 * (size_t)d->ld * (sizeof(S) + sizeof(float));
  const size_t smem2 = 2 * (size_t)d->ld * sizeof(float);
  int t = -1, kind = 0;
  if (want >= NUM_SHAPES + NUM_TMA) { t = want - NUM_SHAPES - NUM_TMA; kind = 2; }
  else if (want >= NUM_SHAPES) { t = want - NUM_SHAPES; kind = 1; }
  // automatic choice, measured on GB300 (FP32): on networks without node locality (random
  // chords, n = 10^4, m = 10^5) the in-sum kind saves the node phase's second read of each F
  // row (264 against 212 iterations/s for the register kind); on renumbered networks (kNN)
  // the register kind's gathers hit L2, and the in-sum kind wins only on long rows (n = 10^4:
  // 235 against 228/s; n = 3000: 1853 against 2672/s). mcf_autotune times every kind on the
  // caller's problem.
  else if (want < 0 &&
           (size_t)d->ld * sizeof(float) >= (d->renumbered ? 32768u : 8192u) &&
           2 * (smem2 + 4096) <= (size_t)smem_optin) {
    for (int c = 0; c < NUM_TMA && t < 0; ++c)
      if (kTmaVpt[c] * TMA_BLOCK >= nchunks) { t = c; kind = 2; }
  }
  if (t < 0) { d->tma = -1; d->tma_kind = 0; d->grid_tma = 0; return MCF_OK; }
  if (kTmaVpt[t] * TMA_BLOCK < nchunks) {
    set_error("shape too small for this problem");
    return MCF_ERR_INVALID;
  }
  const size_t smem = kind == 1 ? smem1 : smem2;
  if (smem + 4096 > (size_t)smem_optin) {
    set_error("rows too long for this shape's shared-memory use");
    return MCF_ERR_INVALID;
  }
  const TmaTable<S>& T = get_tma_table<S>();
  const void* ek = kind == 1 ? (const void*)T.edge[t] : (const void*)T.insum[t];
  CK(cudaFuncSetAttribute(ek, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int on = 0, oe = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&on, (const void*)T.node[t], TMA_NODE_BLOCK, 0));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oe, ek, TMA_BLOCK, smem));
  d->tma = t;
  d->tma_kind = kind;
  d->tma_smem = smem;
  d->grid_tma = std::max(1, std::min(std::max(1, oe) * sms, d->m));
  d->grid_node_pin = std::max(1, std::min(d->n, std::max(1, on) * sms));
  return MCF_OK;
}

template <typename P, typename S>
static int setup_grids(DeviceState* d, int want) {
  const KernelTable<P, S>& T = get_table<P, S>();
  constexpr int VW = StoreTraits<S>::VW;
  const int nchunks = (int)(d->ld / VW);
  const int shape = (want >= 0 && want < NUM_SHAPES) ? want : pick_shape(nchunks);
  if (shape < 0 || T.edge[shape] == nullptr ||
      kShapes[shape].group * kShapes[shape].vpt < nchunks) {
    set_error("no kernel shape covers this problem size at this precision");
    return MCF_ERR_INVALID;
  }
  d->shape = shape;
  d->auto_shape = pick_shape(nchunks);
  const ShapeDesc sd = kShapes[d->shape];
  d->block = sd.block;
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d->device));
  int oe = 0, on = 0, oc = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oe, (const void*)T.edge[d->shape], sd.block, 0));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&on, (const void*)T.node[d->shape], sd.block, 0));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oc, (const void*)T.check[d->shape], sd.block, 0));
  const int gpb = sd.block / sd.group;
  auto grid = [&](int items, int occ) {
    const int need = (items + gpb - 1) / gpb;
    return std::max(1, std::min(need, std::max(1, occ) * sms));
  };
  d->grid_edge = grid(d->m, oe);
  d->grid_node = grid(d->n, on);
  d->grid_check = grid(d->m, oc);
  return MCF_OK;
}


static int configure_shape(DeviceState* d, int want) {
  if (d->precision == MCF_FP64) {
    if (want >= NUM_SHAPES) {
      set_error("the pipelined shapes need FP32 iterates");
      return MCF_ERR_INVALID;
    }
    d->tma = -1;
    return setup_grids<double, double>(d, want);
  }
  int rc;
  if (d->precision == MCF_BF16_F) {
    rc = setup_grids<float, __nv_bfloat16>(d, want);
    if (rc == MCF_OK) rc = setup_tma<__nv_bfloat16>(d, want);
  } else {
    rc = setup_grids<float, float>(d, want);
    if (rc == MCF_OK) rc = setup_tma<float>(d, want);
  }
  return rc;
}

// Head-aligned split of the edge range into at most grid_tma contiguous pieces (edges are
// sorted by head, so a head's in-edges never straddle two CTAs). All CTAs are resident at
// once and the phase ends with the longest piece, so the split minimises the longest one:
// the smallest cap L for which greedy packing of whole heads into pieces of at most L edges
// needs no more than grid_tma pieces (binary search on L; on the n = 10^4, m = 10^5 network
// this gives 1.01 times the mean piece against 1.05 for cuts at multiples of m/grid).
static int upload_cta_ranges(mcf_problem* p, DeviceState* d, cudaStream_t st) {
  if (d->tma < 0) return MCF_OK;
  const int G = d->grid_tma, n = d->n, m = d->m;
  const std::vector<int32_t>& inp = p->topo.in_ptr;
  auto pack = [&](int64_t L, std::vector<int32_t>* ptr) -> int64_t {
    int64_t pieces = 0, cur = 0;
    for (int j = 0; j < n; ++j) {
      const int64_t deg = inp[j + 1] - inp[j];
      if (cur > 0 && cur + deg > L) {
        if (ptr && pieces + 1 <= G) (*ptr)[pieces + 1] = inp[j];
        ++pieces;
        cur = 0;
      }
      cur += deg;
    }
    return pieces + (cur > 0 ? 1 : 0);
  };
  int64_t lo = (m + G - 1) / G, hi = m;
  for (int j = 0; j < n; ++j) lo = std::max<int64_t>(lo, inp[j + 1] - inp[j]);
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (pack(mid, nullptr) <= G) hi = mid; else lo = mid + 1;
  }
  std::vector<int32_t> ptr(G + 1, m);
  ptr[0] = 0;
  pack(lo, &ptr);
  if (d->cta_ptr) {
    cudaDeviceSynchronize();
    dfree(d, d->cta_ptr);
  }
  d->cta_ptr = nullptr;
  if (!dalloc(d, (void**)&d->cta_ptr, (G + 1) * sizeof(int32_t))) {
    set_error("device allocation failed");
    return MCF_ERR_OOM;
  }
  if (!d->Pin && !dalloc(d, &d->Pin, (size_t)n * d->ld * sizeof(float))) {
    set_error("device allocation failed");
    return MCF_ERR_OOM;
  }
  CK(cudaMemcpyAsync(d->cta_ptr, ptr.data(), (G + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  return MCF_OK;
}

// (Re)allocate the per-block partial arrays for the current grids.
static int alloc_partials(DeviceState* d) {
  if (d->part_edge || d->part_node || d->part_check) cudaDeviceSynchronize();
  for (double** b : {&d->part_edge, &d->part_node, &d->part_check})
    if (*b) { dfree(d, *b); *b = nullptr; }
  bool ok = dalloc(d, (void**)&d->part_edge, (size_t)std::max({d->grid_edge, d->grid_tma, 1}) * sizeof(double)) &&
            dalloc(d, (void**)&d->part_node, (size_t)std::max({d->grid_node, d->grid_node_pin, 1}) * NODE_PARTS * sizeof(double)) &&
            dalloc(d, (void**)&d->part_check, (size_t)std::max(d->grid_check, 1) * CHECK_PARTS * sizeof(double));
  if (!ok) {
    set_error("device allocation failed");
    return MCF_ERR_OOM;
  }
  return MCF_OK;
}

static int alloc_state(mcf_problem* p, int precision, int device, int shape, cudaStream_t st_hint,
                       DeviceState** out) {
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    set_error("no CUDA device available (the solver has no CPU path)");
    return MCF_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) {
    set_error("invalid CUDA device ordinal");
    return MCF_ERR_INVALID;
  }
  CK(cudaSetDevice(device));
  DeviceState* d = new DeviceState();
  d->device = device;
  d->precision = precision;
  d->renumbered = !p->topo.node_of.empty();
  d->n = p->n;
  d->m = p->m;
  d->ld = (int)ld_of(p->n);
  d->sbytes = elem_bytes_f(precision);
  d->pbytes = elem_bytes_p(precision);
  int rc = configure_shape(d, shape);
  if (rc != MCF_OK) { free_state(d); return rc; }
  d->requested_shape = shape;
  const size_t n = d->n, m = d->m, ld = d->ld;
  if (cudaStreamCreateWithFlags(&d->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    free_state(d);
    set_error("stream creation failed");
    return MCF_ERR_CUDA;
  }
  d->pool = state_pool(device);
  // pooled allocations are ordered on own_stream; one synchronisation below makes them all
  // usable from any stream
  auto A = [&](void** ptr, size_t bytes) -> bool {
    *ptr = nullptr;
    cudaError_t ea;
    if (d->pool) {
      ea = cudaMallocFromPoolAsync(ptr, bytes, d->pool, d->own_stream);
      if (ea == cudaErrorMemoryAllocation) {   // return the pool's cached memory and retry
        cudaGetLastError();
        cudaStreamSynchronize(d->own_stream);
        cudaMemPoolTrimTo(d->pool, 0);
        ea = cudaMallocFromPoolAsync(ptr, bytes, d->pool, d->own_stream);
      }
    } else {
      ea = cudaMalloc(ptr, bytes);
    }
    if (ea != cudaSuccess) { cudaGetLastError(); *ptr = nullptr; return false; }
    if (!aligned16(*ptr)) { dfree(d, *ptr); *ptr = nullptr; return false; }
    return true;
  };
  bool ok = true;
  for (int i = 0; i < 2 && ok; ++i) ok = A(&d->F[i], m * ld * d->sbytes) && A(&d->Y[i], n * ld * d->pbytes);
  ok = ok && A(&d->Pm, n * ld * d->pbytes) && A(&d->W, n * ld * d->pbytes) &&
       A(&d->That, n * ld * d->pbytes) && A(&d->Uprime, n * ld * d->pbytes) &&
       A(&d->Yhat, n * ld * d->pbytes) && A(&d->mu, 2 * m * d->pbytes) && A(&d->cap, m * d->pbytes);
  if (ok && !p->gamma_mat.empty()) ok = A(&d->G, n * ld * d->pbytes);
  if (ok && precision != MCF_FP64) ok = A(&d->Ylo[0], n * ld * 2) && A(&d->Ylo[1], n * ld * 2);
  ok = ok && A((void**)&d->e_tail, m * 4) && A((void**)&d->e_head, m * 4) &&
       A((void**)&d->in_ptr, (n + 1) * 4) && A((void**)&d->out_ptr, (n + 1) * 4) &&
       A((void**)&d->out_idx, m * 4);
  ok = ok && A((void**)&d->sc, sizeof(DevScalars));
  if (ok && d->pool && cudaStreamSynchronize(d->own_stream) != cudaSuccess) {
    cudaGetLastError();
    ok = false;
  }
  ok = ok && alloc_partials(d) == MCF_OK;
  if (!ok) {
    free_state(d);
    set_error("device allocation failed");
    return MCF_ERR_OOM;
  }
  if (cudaMallocHost((void**)&d->sc_host, sizeof(DevScalars)) != cudaSuccess) {
    cudaGetLastError();
    free_state(d);
    set_error("pinned host allocation failed");
    return MCF_ERR_OOM;
  }
  cudaStream_t st = st_hint ? st_hint : d->own_stream;
  const Topology& t = p->topo;
  CK(cudaMemcpyAsync(d->e_tail, t.e_tail.data(), m * 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d->e_head, t.e_head.data(), m * 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d->in_ptr, t.in_ptr.data(), (n + 1) * 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d->out_ptr, t.out_ptr.data(), (n + 1) * 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d->out_idx, t.out_idx.data(), m * 4, cudaMemcpyHostToDevice, st));
  // the kernels read every chunk of every row, so pads must start at zero everywhere
  for (void* b : {d->That, d->Uprime, d->Yhat}) CK(cudaMemsetAsync(b, 0, n * ld * d->pbytes, st));
  CK(cudaStreamSynchronize(st));
  rc = upload_cta_ranges(p, d, st);
  if (rc != MCF_OK) { free_state(d); return rc; }
  p->data_dirty = true;
  *out = d;
  return MCF_OK;
}

void device_free(mcf_problem* p) {
  free_state(p->ds);
  p->ds = nullptr;
}

// ------------------------------------------------------------------ iteration

template <typename P, typename S>
static IterArgs<P, S> make_args(DeviceState* d, const mcf_problem* p, double rho, bool lo) {
  IterArgs<P, S> a{};
  a.n = d->n;
  a.m = d->m;
  a.ld = d->ld;
  a.e_tail = d->e_tail;
  a.e_head = d->e_head;
  a.in_ptr = d->in_ptr;
  a.out_ptr = d->out_ptr;
  a.out_idx = d->out_idx;
  a.cap = (const P*)d->cap;
  a.F[0] = (S*)d->F[0];
  a.F[1] = (S*)d->F[1];
  a.Y[0] = (P*)d->Y[0];
  a.Y[1] = (P*)d->Y[1];
  a.Ylo[0] = lo ? (__nv_bfloat16*)d->Ylo[0] : nullptr;
  a.Ylo[1] = lo ? (__nv_bfloat16*)d->Ylo[1] : nullptr;
  a.Pm = (P*)d->Pm;
  a.W = (const P*)d->W;
  a.Gm = (const P*)d->G;
  a.gamma = (P)p->gamma_scalar;
  a.kind = p->kind;
  a.mu = (P*)d->mu;
  a.mu_lo = (P*)d->mu + d->m;
  a.That = (P*)d->That;
  a.Uprime = (P*)d->Uprime;
  a.Yhat = (P*)d->Yhat;
  a.part_edge = d->part_edge;
  a.part_node = d->part_node;
  a.part_check = d->part_check;
  a.sc = d->sc;
  a.rho = (P)rho;
  a.Pin = (P*)d->Pin;
  a.cta_ptr = d->cta_ptr;
  return a;
}

// Edge and node phase launches of one iteration (register shapes or the pipelined pair).
template <typename P, typename S>
static cudaError_t launch_phase(DeviceState* d, void** kargs, int which, bool check, cudaStream_t st) {
  if constexpr (!std::is_same<P, double>::value) {
    if (d->tma >= 0) {
      const TmaTable<S>& T = get_tma_table<S>();
      if (which == 0)
        return cudaLaunchKernel(d->tma_kind == 1 ? (const void*)T.edge[d->tma] : (const void*)T.insum[d->tma],
                                dim3(d->grid_tma), dim3(TMA_BLOCK), kargs, d->tma_smem, st);
      return cudaLaunchKernel(check ? (const void*)T.node_chk[d->tma] : (const void*)T.node[d->tma],
                              dim3(d->grid_node_pin), dim3(TMA_NODE_BLOCK), kargs, 0, st);
    }
  }
  const KernelTable<P, S>& T = get_table<P, S>();
  if (which == 0)
    return cudaLaunchKernel((const void*)T.edge[d->shape], dim3(d->grid_edge), dim3(d->block), kargs, 0, st);
  return cudaLaunchKernel(check ? (const void*)T.node_chk[d->shape] : (const void*)T.node[d->shape],
                          dim3(d->grid_node), dim3(d->block), kargs, 0, st);
}

static int edge_blocks(const DeviceState* d) { return d->tma >= 0 ? d->grid_tma : d->grid_edge; }
static int node_blocks(const DeviceState* d) { return d->tma >= 0 ? d->grid_node_pin : d->grid_node; }

template <typename P, typename S>
static cudaError_t launch_iteration(DeviceState* d, IterArgs<P, S> a, int parity, bool check,
                                    cudaStream_t st) {
  const KernelTable<P, S>& T = get_table<P, S>();
  a.parity = parity;
  a.check = check ? 1 : 0;
  void* kargs[] = {&a};
  cudaError_t e;
  e = launch_phase<P, S>(d, kargs, 0, check, st);
  if (e != cudaSuccess) return e;
  e = launch_phase<P, S>(d, kargs, 1, check, st);
  if (e != cudaSuccess) return e;
  if (check) {
    e = cudaLaunchKernel((const void*)T.check[d->shape], dim3(d->grid_check), dim3(d->block), kargs, 0, st);
    if (e != cudaSuccess) return e;
  }
  ScalarArgs sa{d->sc, d->part_edge, edge_blocks(d), d->part_node, node_blocks(d),
                d->part_check, d->grid_check, check ? 1 : 0};
  scalar_kernel<<<1, 256, 0, st>>>(sa);
  return cudaGetLastError();
}

// One iteration with a CUDA event before the first and after every kernel (on st).
struct EventPool {
  std::vector<cudaEvent_t> ev;
  std::vector<int> kind;   // kernel kind that ends at event i (i >= 1)
  size_t used = 0;
  cudaEvent_t next(int k) {
    if (used == ev.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      ev.push_back(e);
      kind.push_back(-1);
    }
    kind[used] = k;
    return ev[used++];
  }
  ~EventPool() {
    for (auto e : ev) cudaEventDestroy(e);
  }
};

template <typename P, typename S>
static cudaError_t launch_iteration_timed(DeviceState* d, IterArgs<P, S> a, int parity, bool check,
                                          cudaStream_t st, EventPool& pool) {
  const KernelTable<P, S>& T = get_table<P, S>();
  a.parity = parity;
  a.check = check ? 1 : 0;
  void* kargs[] = {&a};
  cudaError_t e;
  if (pool.used == 0) cudaEventRecord(pool.next(-1), st);
  {
    NvtxRange r("pdmcf edge phase");
    e = launch_phase<P, S>(d, kargs, 0, check, st);
  }
  if (e != cudaSuccess) return e;
  cudaEventRecord(pool.next(0), st);
  {
    NvtxRange r("pdmcf node phase");
    e = launch_phase<P, S>(d, kargs, 1, check, st);
  }
  if (e != cudaSuccess) return e;
  cudaEventRecord(pool.next(1), st);
  if (check) {
    NvtxRange r("pdmcf check phase");
    e = cudaLaunchKernel((const void*)T.check[d->shape], dim3(d->grid_check), dim3(d->block), kargs, 0, st);
    if (e != cudaSuccess) return e;
    cudaEventRecord(pool.next(2), st);
  }
  ScalarArgs sa{d->sc, d->part_edge, edge_blocks(d), d->part_node, node_blocks(d),
                d->part_check, d->grid_check, check ? 1 : 0};
  scalar_kernel<<<1, 256, 0, st>>>(sa);
  cudaEventRecord(pool.next(3), st);
  return cudaGetLastError();
}

// Add the event intervals of a synchronized chunk to kt and reset the pool.
static void drain_events(EventPool& pool, mcf_kernel_times* kt) {
  for (size_t i = 1; i < pool.used; ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, pool.ev[i - 1], pool.ev[i]);
    kt->ms[pool.kind[i]] += ms;
    kt->launches[pool.kind[i]] += 1;
    kt->ms_total += ms;
  }
  pool.used = 0;
}

// Capture k_check iterations starting at the given parity, the last one a check.
template <typename P, typename S>
static bool capture_chunk(DeviceState* d, const IterArgs<P, S>& a, int parity, int len,
                          cudaStream_t st, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  bool ok = true;
  int par = parity;
  for (int i = 0; i < len && ok; ++i) {
    ok = launch_iteration<P, S>(d, a, par, i == len - 1, st) == cudaSuccess;
    par ^= 1;
  }
  const cudaError_t e = cudaStreamEndCapture(st, &g);
  if (!ok || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return false;
  }
  const cudaError_t ei = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

static void fill_scalars(const DevScalars& s, const mcf_problem* p, mcf_result* res) {
  res->iters = s.k;
  res->feasible = s.feasible;
  res->utility = s.P;
  res->dual_bound = s.D;
  res->r = s.r;
  res->r_over_nm = s.r / ((double)p->n * (double)p->m);
  res->rel_gap = s.rel_gap;
  res->rel_cons = s.rel_cons;
  res->rel_stat = s.rel_stat;
  res->rel_kkt = s.rel_kkt;
  res->nonpos_frac = s.nonpos_frac;
  res->omega = s.omega;
  res->delta_f = s.dF;
  res->delta_y = s.dY;
  res->omega_frozen_at = (s.freeze >= 0 && s.freeze <= s.k) ? s.freeze : -1;
}

// Extra stop rules of the BF16 phase that precedes an FP32 polish: hand off once the
// relative KKT is within `handoff` of the target, or when it has not improved by 5 % over
// `stall_checks` consecutive checks (BF16 rounding of F sets a floor on the accuracy).
struct PhaseRule {
  double handoff = 0.0;
  int stall_checks = 0;
  bool skip_outputs = false;
};

// mcf_options.check_log: one JSON line per stop test (Sec. 3.1's convergence diagnostics).
struct CheckLog {
  FILE* f = nullptr;
  explicit CheckLog(const char* path) { if (path && *path) f = std::fopen(path, "a"); }
  ~CheckLog() { if (f) std::fclose(f); }
};

static void json_num(FILE* f, const char* key, double v, bool last = false) {
  if (std::isfinite(v)) std::fprintf(f, "\"%s\": %.17g%s", key, v, last ? "" : ", ");
  else std::fprintf(f, "\"%s\": null%s", key, last ? "" : ", ");
}

static void write_check_line(FILE* f, const DevScalars& h, int n, int m, int precision) {
  std::fprintf(f, "{\"k\": %lld, ", (long long)h.k);
  json_num(f, "omega", h.omega);
  json_num(f, "r_over_nm", h.r / ((double)n * (double)m));
  json_num(f, "rel_kkt", h.rel_kkt);
  json_num(f, "rel_gap", h.rel_gap);
  json_num(f, "rel_cons", h.rel_cons);
  json_num(f, "rel_stat", h.rel_stat);
  json_num(f, "utility", h.P);
  json_num(f, "dual_bound", h.D);
  json_num(f, "nonpos_frac", h.nonpos_frac);
  std::fprintf(f, "\"omega_adapting\": %s, \"precision\": \"%s\"}\n",
               (h.freeze >= 0 && h.freeze <= h.k) ? "false" : "true",
               precision == MCF_FP64 ? "fp64" : (precision == MCF_BF16_F ? "bf16" : "fp32"));
  std::fflush(f);
}

// mcf_test_withhold_next_copy: one pending request, taken by the next solve that runs the
// bulk-copy edge phase.
static std::atomic<int> g_withhold_request{0};
static bool take_withhold_request() { return g_withhold_request.exchange(0) != 0; }

template <typename P, typename S>
static int solve_t(mcf_problem* p, DeviceState* d, const mcf_options* o, mcf_result* res,
                   cudaStream_t st, mcf_kernel_times* kt, const PhaseRule& rule = PhaseRule()) {
  const int n = d->n;
  const size_t ld = d->ld, m = d->m;
  if (p->data_dirty) {
    int rc = upload_data<P>(p, d, st);
    if (rc != MCF_OK) return rc;
  }
  const bool warm = o->warm_start && d->valid;
  DevScalars& h = *d->sc_host;
  if (!warm) {
    d->cur = 0;
    CK(cudaMemsetAsync(d->F[0], 0, m * ld * d->sbytes, st));
    CK(cudaMemsetAsync(d->F[1], 0, m * ld * d->sbytes, st));
    CK(cudaMemsetAsync(d->Pm, 0, (size_t)n * ld * d->pbytes, st));
    CK(cudaMemsetAsync(d->mu, 0, 2 * m * d->pbytes, st));
    init_y_kernel<P><<<1024, 256, 0, st>>>((P*)d->Y[0], n, (int)ld);
    CK(cudaGetLastError());
    p->omega = o->omega0 > 0 ? o->omega0 : 1.0;
  }
  std::memset(&h, 0, sizeof(DevScalars));
  h.eta = p->eta;
  h.omega = p->omega;
  h.alpha = h.eta / h.omega;
  h.beta = h.eta * h.omega;
  h.alpha_last = h.alpha;
  h.beta_last = h.beta;
  h.k = 0;
  h.theta = o->theta;
  h.tau = o->tau;
  h.k_adapt = o->k_adapt > 0 ? o->k_adapt : 1;
  h.freeze = o->omega_freeze_iter;
  h.guard = o->adapt_guard;
  h.guard_below = o->adapt_guard_below;
  h.omega_ref = 0.0;
  h.omega_arm = 0.0;
  h.best_kkt = INFINITY;
  h.r = INFINITY;
  h.rel_kkt = INFINITY;
  h.n = n;
  h.m = (int)m;
  CK(cudaMemcpyAsync(d->sc, &h, sizeof(DevScalars), cudaMemcpyHostToDevice, st));

  const bool lo = o->compensated_duals && d->Ylo[0] != nullptr;
  if (lo && (!warm || !d->lo_live)) {
    CK(cudaMemsetAsync(d->Ylo[0], 0, (size_t)n * ld * 2, st));
    CK(cudaMemsetAsync(d->Ylo[1], 0, (size_t)n * ld * 2, st));
  }
  d->lo_live = lo;
  const IterArgs<P, S> args = make_args<P, S>(d, p, o->rho, lo);
  // testing aid (mcf_test_withhold_next_copy): the first edge launch of this solve withholds
  // block 0's first bulk copies, so its bounded wait runs out and the solve reports it
  const bool withhold = d->tma >= 0 && d->tma_kind == 1 && take_withhold_request();
  IterArgs<P, S> args_w = args;
  args_w.withhold = 1;
  const int64_t max_iters = o->max_iters;
  const int kc = std::max(1, o->k_check);
  bool use_graphs = o->use_graphs && !d->graphs_broken && kt == nullptr;
  EventPool pool;
  if (kt) {
    std::memset(kt, 0, sizeof(*kt));
    kt->shape = d->tma < 0 ? d->shape : NUM_SHAPES + (d->tma_kind == 2 ? NUM_TMA : 0) + d->tma;
  }
  if (use_graphs && (d->graph_len != kc || d->graph_rho != o->rho || d->graph_stream != st ||
                     d->graph_lo != lo)) {
    destroy_graphs(d);
    d->graph_len = kc;
    d->graph_rho = o->rho;
    d->graph_stream = st;
    d->graph_lo = lo;
  }
  int parity = d->cur;
  CheckLog log_file(o->check_log);
  FILE* log = log_file.f;
  if (o->check_log && *o->check_log && !log) {
    set_error(std::string("cannot open the check log ") + o->check_log);
    return MCF_ERR_INVALID;
  }
  int64_t k = 0;
  double best_kkt = INFINITY;
  int since_best = 0;
  double floor_best = INFINITY;
  int floor_since = 0;
  bool floor_frozen = false;   // omega had stopped adapting when the count last restarted
  bool stalled = false;
  int status = MCF_ERR_NOT_CONVERGED;
  if (o->stop_mode == MCF_STOP_NONE) status = MCF_OK;
  bool any = false;
  NvtxRange solve_range(d->precision == MCF_FP64 ? "pdmcf solve fp64"
                        : d->precision == MCF_BF16_F ? "pdmcf solve bf16" : "pdmcf solve fp32");
  while (k < max_iters) {
    NvtxRange chunk_range("pdmcf chunk");
    const int64_t chunk = std::min<int64_t>(kc - (k % kc), max_iters - k);
    const bool stall_first = withhold && k == 0;
    if (use_graphs && chunk == kc && !stall_first) {
      if (!d->graph[parity] && !capture_chunk<P, S>(d, args, parity, kc, st, &d->graph[parity])) {
        d->graphs_broken = true;
        use_graphs = false;
      }
    }
    if (use_graphs && chunk == kc && !stall_first) {
      CK(cudaGraphLaunch(d->graph[parity], st));
      if (kc & 1) parity ^= 1;
    } else {
      for (int64_t i = 0; i < chunk; ++i) {
        const IterArgs<P, S>& ai = (stall_first && i == 0) ? args_w : args;
        if (kt) CK((launch_iteration_timed<P, S>(d, ai, parity, i == chunk - 1, st, pool)));
        else CK((launch_iteration<P, S>(d, ai, parity, i == chunk - 1, st)));
        parity ^= 1;
      }
    }
    CK(cudaMemcpyAsync(d->sc_host, d->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (kt) drain_events(pool, kt);
    k += chunk;
    any = true;
    d->cur = parity;
    d->valid = true;
    if (log) write_check_line(log, h, n, m, d->precision);
    if (h.wait_timeout) {
      set_error("a bounded device-side wait timed out; the iteration was abandoned");
      d->valid = false;
      return MCF_ERR_CUDA;
    }
    if (h.numeric_error) {
      status = MCF_ERR_NUMERIC;
      set_error("NaN or Inf in the iterates");
      break;
    }
    if (o->stop_mode == MCF_STOP_PAPER && h.r < (double)n * (double)m * o->eps) { status = MCF_OK; break; }
    if (o->stop_mode == MCF_STOP_REL_KKT && h.rel_kkt < o->eps) { status = MCF_OK; break; }
    if (rule.handoff > 0.0 && h.rel_kkt < rule.handoff) break;
    if (o->stop_mode == MCF_STOP_REL_KKT && o->stall_checks > 0 && h.rel_kkt < 100.0 * o->eps) {
      const bool frozen = h.freeze >= 0 && h.freeze <= h.k;
      if (frozen != floor_frozen) { floor_frozen = frozen; floor_best = INFINITY; floor_since = 0; }
      if (h.rel_kkt < 0.95 * floor_best) { floor_best = h.rel_kkt; floor_since = 0; }
      else if (++floor_since >= o->stall_checks) { stalled = true; break; }
    }
    if (rule.stall_checks > 0) {
      if (h.rel_kkt < 0.95 * best_kkt) { best_kkt = h.rel_kkt; since_best = 0; }
      else if (++since_best >= rule.stall_checks) break;
    }
  }
  p->omega = h.omega;
  if (!any) {
    set_error("max_iters must be >= 1");
    return MCF_ERR_INVALID;
  }
  fill_scalars(h, p, res);
  res->status = status;
  res->stalled = stalled ? 1 : 0;
  if (!rule.skip_outputs && (res->T || res->Y || res->F)) {
    int rc = device_copy_outputs(p, res);
    if (rc != MCF_OK) return rc;
  }
  return status;
}

template <typename P, typename S>
static int copy_outputs_t(mcf_problem* p, DeviceState* d, mcf_result* res, cudaStream_t st) {
  const int n = d->n, m = d->m;
  const size_t ld = d->ld;
  int rc = ensure_node_map(p, d, st);
  if (rc != MCF_OK) return rc;
  // out[r][c] = in[rowmap[c]][colmap[r]] in chunks of rows, through a device stage
  auto gather = [&](const P* in, const int32_t* rowmap, int nrows, int ncols, double* out) -> int {
    const int rows = chunk_rows(nrows, ncols);
    double* stage = nullptr;
    if (!salloc(d, (void**)&stage, (size_t)rows * ncols * sizeof(double), st)) {
      set_error("device allocation for an output failed");
      return MCF_ERR_OOM;
    }
    cudaError_t e = cudaSuccess;
    for (int r0 = 0; r0 < nrows && e == cudaSuccess; r0 += rows) {
      const int nr = std::min(rows, nrows - r0);
      const dim3 grid((ncols + 31) / 32, (nr + 31) / 32);
      gather_out_kernel<P><<<grid, dim3(32, 8), 0, st>>>(in, ld, rowmap, d->node_map, stage, r0,
                                                         nr, ncols);
      e = cudaGetLastError();
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(out + (size_t)r0 * ncols, stage, (size_t)nr * ncols * sizeof(double),
                            cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    sfree(d, stage, st);
    CK(e);
    return MCF_OK;
  };
  prefault_host(res->T, (size_t)n * n * sizeof(double));
  prefault_host(res->Y, (size_t)n * n * sizeof(double));
  prefault_host(res->F, (size_t)n * m * sizeof(double));
  // T[i][j] = That[node(j)][node(i)], Y likewise: row map node, column map node
  if (res->T && (rc = gather((const P*)d->That, d->node_map, n, n, res->T)) != MCF_OK) return rc;
  if (res->Y && (rc = gather((const P*)d->Yhat, d->node_map, n, n, res->Y)) != MCF_OK) return rc;
  if (res->F) {
    // F[i][l] = F^[internal edge of l][node(i)]
    P* tmp = nullptr;
    int32_t* emap = nullptr;
    if (!salloc(d, (void**)&tmp, (size_t)m * ld * sizeof(P), st) ||
        !salloc(d, (void**)&emap, (size_t)m * 4, st)) {
      sfree(d, tmp, st);
      set_error("device allocation for the F output failed");
      return MCF_ERR_OOM;
    }
    std::vector<int32_t> inv(m);
    for (int e2 = 0; e2 < m; ++e2) inv[p->topo.perm[e2]] = e2;
    cudaError_t e = cudaMemcpyAsync(emap, inv.data(), (size_t)m * 4, cudaMemcpyHostToDevice, st);
    const int prev = d->cur ^ 1;   // F^{k-3/2} and Y^{k-1} of the last iteration
    if (e == cudaSuccess) {
      fhat_kernel<P, S><<<2048, 256, 0, st>>>((const S*)d->F[prev], (const P*)d->Y[prev],
                                             d->lo_live ? (const __nv_bfloat16*)d->Ylo[prev] : nullptr,
                                             d->e_tail, d->e_head, (const P*)d->mu,
                                             (const P*)d->mu + m, d->sc, tmp, m, (int)ld);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // inv dies at return
    rc = e == cudaSuccess ? gather(tmp, emap, n, m, res->F) : MCF_ERR_CUDA;
    if (e != cudaSuccess) set_error(std::string("CUDA error ") + cudaGetErrorString(e));
    sfree(d, tmp, st);
    sfree(d, emap, st);
    if (rc != MCF_OK) return rc;
  }
  return MCF_OK;
}

}  // namespace pdmcf

extern "C" int mcf_test_withhold_next_copy(void) {
  pdmcf::g_withhold_request.store(1);
  return MCF_OK;
}

extern "C" int mcf_shape_info(int* group, int* vpt, int* block, int* kind) {
  using namespace pdmcf;
  for (int s = 0; s < NUM_SHAPES + 2 * NUM_TMA; ++s) {
    const int k = s < NUM_SHAPES ? 0 : (s < NUM_SHAPES + NUM_TMA ? 1 : 2);
    const int t = k == 0 ? 0 : (s - NUM_SHAPES) % NUM_TMA;
    if (group) group[s] = k ? TMA_BLOCK : kShapes[s].group;
    if (vpt) vpt[s] = k ? kTmaVpt[t] : kShapes[s].vpt;
    if (block) block[s] = k ? TMA_BLOCK : kShapes[s].block;
    if (kind) kind[s] = k;
  }
  return NUM_SHAPES + 2 * NUM_TMA;
}

namespace pdmcf {

int device_copy_outputs(mcf_problem* p, mcf_result* res) {
  DeviceState* d = p->ds;
  if (!d || !d->valid) {
    set_error("no solution resident on the device");
    return MCF_ERR_INVALID;
  }
  CK(cudaSetDevice(d->device));
  cudaStream_t st = d->own_stream;
  if (d->precision == MCF_FP64) return copy_outputs_t<double, double>(p, d, res, st);
  if (d->precision == MCF_BF16_F) return copy_outputs_t<float, __nv_bfloat16>(p, d, res, st);
  return copy_outputs_t<float, float>(p, d, res, st);
}

__global__ void bf16_to_f32_kernel(const __nv_bfloat16* src, float* dst, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = __bfloat162float(src[i]);
}

// Move the resident iterate of a BF16-storage state into a fresh FP32 state on the device:
// F^{k-1/2} widened exactly, Y^k, P = F^{k-1/2} A^T and the projection multipliers copied.
static int transfer_to_fp32(mcf_problem* p, const mcf_options* o, cudaStream_t st) {
  DeviceState* src = p->ds;
  DeviceState* dst = nullptr;
  int rc = alloc_state(p, MCF_FP32, src->device, o->shape, (cudaStream_t)o->cuda_stream, &dst);
  if (rc != MCF_OK) return rc;
  dst->requested_shape = o->shape;
  const size_t n = src->n, m = src->m, ld = src->ld;
  const int c = src->cur;
  bf16_to_f32_kernel<<<2048, 256, 0, st>>>((const __nv_bfloat16*)src->F[c], (float*)dst->F[c], m * ld);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(dst->Y[c], src->Y[c], n * ld * 4, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dst->Pm, src->Pm, n * ld * 4, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dst->mu, src->mu, 2 * m * 4, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && src->lo_live)
    e = cudaMemcpyAsync(dst->Ylo[c], src->Ylo[c], n * ld * 2, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    free_state(dst);
    set_error(std::string("CUDA error ") + cudaGetErrorString(e));
    return MCF_ERR_CUDA;
  }
  dst->cur = c;
  dst->valid = true;
  dst->lo_live = src->lo_live;
  free_state(src);
  p->ds = dst;
  p->data_dirty = true;
  return MCF_OK;
}

// ------------------------------------------------------------------ batched-engine hooks

// FP32 state on o->device for a batched run: cold start (F = 0, Y = I - 11^T, P = 0,
// mu = 0, omega = omega0) unless a warm start is asked for and an iterate is resident.
int batch_prepare_state(mcf_problem* p, const mcf_options* o, cudaStream_t st, bool* warm) {
  if (p->ds && (p->ds->precision != MCF_FP32 || p->ds->device != o->device)) device_free(p);
  if (!p->ds) {
    int rc = alloc_state(p, MCF_FP32, o->device, -1, st, &p->ds);
    if (rc != MCF_OK) return rc;
  }
  DeviceState* d = p->ds;
  if (p->data_dirty) {
    int rc = upload_data<float>(p, d, st);
    if (rc != MCF_OK) return rc;
  }
  *warm = o->warm_start && d->valid;
  const size_t n = d->n, m = d->m, ld = d->ld;
  const bool lo = o->compensated_duals && d->Ylo[0] != nullptr;
  if (lo && (!*warm || !d->lo_live)) {
    CK(cudaMemsetAsync(d->Ylo[0], 0, n * ld * 2, st));
    CK(cudaMemsetAsync(d->Ylo[1], 0, n * ld * 2, st));
  }
  d->lo_live = lo;
  if (!*warm) {
    d->cur = 0;
    CK(cudaMemsetAsync(d->F[0], 0, m * ld * 4, st));
    CK(cudaMemsetAsync(d->F[1], 0, m * ld * 4, st));
    CK(cudaMemsetAsync(d->Pm, 0, n * ld * 4, st));
    CK(cudaMemsetAsync(d->mu, 0, 2 * m * 4, st));
    init_y_kernel<float><<<1024, 256, 0, st>>>((float*)d->Y[0], (int)n, (int)ld);
    CK(cudaGetLastError());
    p->omega = o->omega0 > 0 ? o->omega0 : 1.0;
  }
  CK(cudaStreamSynchronize(st));
  d->valid = false;   // the iterate is in flux until the engine hands it back
  return MCF_OK;
}

void batch_state_pointers(mcf_problem* p, BatchInst* bi, int* parity) {
  DeviceState* d = p->ds;
  *parity = d->cur;
  bi->n = d->n;
  bi->m = d->m;
  bi->ld = d->ld;
  bi->kind = p->kind;
  bi->gamma = (float)p->gamma_scalar;
  bi->e_tail = d->e_tail;
  bi->e_head = d->e_head;
  bi->in_ptr = d->in_ptr;
  bi->out_ptr = d->out_ptr;
  bi->out_idx = d->out_idx;
  bi->cap = (const float*)d->cap;
  bi->W = (const float*)d->W;
  bi->Gm = (const float*)d->G;
  bi->F[0] = (float*)d->F[0];
  bi->F[1] = (float*)d->F[1];
  bi->Y[0] = (float*)d->Y[0];
  bi->Y[1] = (float*)d->Y[1];
  bi->Ylo[0] = d->lo_live ? (__nv_bfloat16*)d->Ylo[0] : nullptr;
  bi->Ylo[1] = d->lo_live ? (__nv_bfloat16*)d->Ylo[1] : nullptr;
  bi->Pm = (float*)d->Pm;
  bi->mu = (float*)d->mu;
  bi->mu_lo = (float*)d->mu + d->m;
  bi->That = (float*)d->That;
  bi->Uprime = (float*)d->Uprime;
  bi->Yhat = (float*)d->Yhat;
}

// The engine's final scalars become the problem's resident state (warm starts, outputs).
void batch_finish_state(mcf_problem* p, int parity, const DevScalars& s, cudaStream_t st) {
  DeviceState* d = p->ds;
  d->cur = parity;
  d->valid = true;
  p->omega = s.omega;
  cudaMemcpyAsync(d->sc, &s, sizeof(DevScalars), cudaMemcpyHostToDevice, st);
  cudaStreamSynchronize(st);
}

// ------------------------------------------------------------------ warm-state checkpoint
// The resident warm tuple of Sec. 3.1 (F^{k-1/2}, Y^k with its compensated tail, the state
// P = F^{k-1/2} A^T of the relaxation identity, the projection multipliers and omega) in the
// device layout and internal numbering, written to or read from a host file through a
// 64 MB pinned staging buffer.

namespace {
struct StateHeader {
  char magic[8];          // "PDMCFWS1"
  int32_t version;        // 1
  int32_t n, m, ld, precision, lo_live;
  double omega;
  uint64_t topo_hash;     // FNV-1a over the internal (tail, head) order
  uint64_t bytes[5];      // F, Y, Y tail, P, mu
};

uint64_t topo_hash(const Topology& t) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](const std::vector<int32_t>& v) {
    for (int32_t x : v)
      for (int b = 0; b < 4; ++b) { h ^= (uint64_t)((x >> (8 * b)) & 0xff); h *= 1099511628211ull; }
  };
  mix(t.e_tail);
  mix(t.e_head);
  mix(t.node_of);
  return h;
}

constexpr size_t kStage = (size_t)64 << 20;
}  // namespace

int device_save_state(mcf_problem* p, const char* path) {
  DeviceState* d = p->ds;
  if (!d || !d->valid) {
    set_error("the problem has no solved state to save");
    return MCF_ERR_INVALID;
  }
  CK(cudaSetDevice(d->device));
  const size_t n = d->n, m = d->m, ld = d->ld;
  StateHeader h{};
  std::memcpy(h.magic, "PDMCFWS1", 8);
  h.version = 1;
  h.n = d->n; h.m = d->m; h.ld = d->ld; h.precision = d->precision;
  h.lo_live = d->lo_live ? 1 : 0;
  h.omega = p->omega;
  h.topo_hash = topo_hash(p->topo);
  const void* src[5] = {d->F[d->cur], d->Y[d->cur], d->lo_live ? d->Ylo[d->cur] : nullptr, d->Pm, d->mu};
  const uint64_t bytes[5] = {m * ld * d->sbytes, n * ld * d->pbytes, d->lo_live ? n * ld * 2 : 0,
                             n * ld * d->pbytes, 2 * m * d->pbytes};
  std::memcpy(h.bytes, bytes, sizeof(bytes));
  FILE* f = std::fopen(path, "wb");
  if (!f) {
    set_error(std::string("cannot open ") + path + " for writing");
    return MCF_ERR_INVALID;
  }
  char* stage = nullptr;
  if (cudaMallocHost((void**)&stage, kStage) != cudaSuccess) {
    std::fclose(f);
    cudaGetLastError();
    set_error("pinned host allocation failed");
    return MCF_ERR_OOM;
  }
  bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1;
  cudaError_t e = cudaDeviceSynchronize();   // the state is complete only after the solve
  for (int a = 0; a < 5 && ok && e == cudaSuccess; ++a)
    for (uint64_t off = 0; off < bytes[a] && ok && e == cudaSuccess; off += kStage) {
      const size_t len = (size_t)std::min<uint64_t>(kStage, bytes[a] - off);
      e = cudaMemcpy(stage, (const char*)src[a] + off, len, cudaMemcpyDeviceToHost);
      ok = e == cudaSuccess && std::fwrite(stage, 1, len, f) == len;
    }
  cudaFreeHost(stage);
  const bool closed = std::fclose(f) == 0;
  if (e != cudaSuccess) {
    set_error(std::string("CUDA error ") + cudaGetErrorString(e) + " while saving the state");
    return MCF_ERR_CUDA;
  }
  if (!ok || !closed) {
    set_error(std::string("write to ") + path + " failed");
    return MCF_ERR_INVALID;
  }
  return MCF_OK;
}

int device_load_state(mcf_problem* p, const char* path, int device) {
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    set_error(std::string("cannot open ") + path);
    return MCF_ERR_INVALID;
  }
  StateHeader h{};
  if (std::fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, "PDMCFWS1", 8) != 0 ||
      h.version != 1) {
    std::fclose(f);
    set_error(std::string(path) + " is not a PDMCF warm-state file");
    return MCF_ERR_INVALID;
  }
  if (h.n != p->n || h.m != p->m || h.ld != (int)ld_of(p->n) || h.topo_hash != topo_hash(p->topo) ||
      (h.precision != MCF_FP32 && h.precision != MCF_FP64 && h.precision != MCF_BF16_F)) {
    std::fclose(f);
    set_error("the saved state belongs to a different network");
    return MCF_ERR_INVALID;
  }
  if (p->ds && (p->ds->precision != h.precision || p->ds->device != device)) device_free(p);
  if (!p->ds) {
    int rc = alloc_state(p, h.precision, device, -1, nullptr, &p->ds);
    if (rc != MCF_OK) { std::fclose(f); return rc; }
  }
  DeviceState* d = p->ds;
  CK(cudaSetDevice(d->device));
  const size_t n = d->n, m = d->m, ld = d->ld;
  const uint64_t want[5] = {m * ld * d->sbytes, n * ld * d->pbytes, h.lo_live ? n * ld * 2 : 0,
                            n * ld * d->pbytes, 2 * m * d->pbytes};
  if (std::memcmp(want, h.bytes, sizeof(want)) != 0 || (h.lo_live && !d->Ylo[0])) {
    std::fclose(f);
    set_error("the saved state's array sizes do not match this problem");
    return MCF_ERR_INVALID;
  }
  void* dst[5] = {d->F[0], d->Y[0], h.lo_live ? d->Ylo[0] : nullptr, d->Pm, d->mu};
  char* stage = nullptr;
  if (cudaMallocHost((void**)&stage, kStage) != cudaSuccess) {
    std::fclose(f);
    cudaGetLastError();
    set_error("pinned host allocation failed");
    return MCF_ERR_OOM;
  }
  d->valid = false;
  bool ok = true;
  cudaError_t e = cudaDeviceSynchronize();
  for (int a = 0; a < 5 && ok && e == cudaSuccess; ++a)
    for (uint64_t off = 0; off < want[a] && ok && e == cudaSuccess; off += kStage) {
      const size_t len = (size_t)std::min<uint64_t>(kStage, want[a] - off);
      ok = std::fread(stage, 1, len, f) == len;
      if (ok) e = cudaMemcpy((char*)dst[a] + off, stage, len, cudaMemcpyHostToDevice);
    }
  cudaFreeHost(stage);
  std::fclose(f);
  if (e != cudaSuccess) {
    set_error(std::string("CUDA error ") + cudaGetErrorString(e) + " while loading the state");
    return MCF_ERR_CUDA;
  }
  if (!ok) {
    set_error(std::string(path) + " is truncated");
    return MCF_ERR_INVALID;
  }
  d->cur = 0;
  d->lo_live = h.lo_live != 0;
  d->valid = true;
  p->omega = h.omega;
  return MCF_OK;
}

int device_solve(mcf_problem* p, const mcf_options* o, mcf_result* res, mcf_kernel_times* kt) {
  const int prec = o->precision;
  if (prec != MCF_FP32 && prec != MCF_FP64 && prec != MCF_BF16_F) {
    set_error("unknown precision");
    return MCF_ERR_INVALID;
  }
  cudaStream_t user = (cudaStream_t)o->cuda_stream;
  if (p->ds && (p->ds->precision != prec || p->ds->device != o->device)) device_free(p);
  if (!p->ds) {
    int rc = alloc_state(p, prec, o->device, o->shape, user, &p->ds);
    if (rc != MCF_OK) return rc;
  }
  DeviceState* d = p->ds;
  CK(cudaSetDevice(d->device));
  if (o->shape != d->requested_shape) {
    // a different launch shape: new grids and partial arrays, same resident iterate
    int rc = configure_shape(d, o->shape);
    if (rc == MCF_OK) rc = alloc_partials(d);
    if (rc == MCF_OK) rc = upload_cta_ranges(p, d, user ? user : d->own_stream);
    if (rc != MCF_OK) return rc;
    d->requested_shape = o->shape;
    destroy_graphs(d);
  }
  cudaStream_t st = user ? user : d->own_stream;
  if (prec == MCF_FP64) return solve_t<double, double>(p, d, o, res, st, kt);
  if (prec == MCF_BF16_F) {
    if (o->polish_iters <= 0) return solve_t<float, __nv_bfloat16>(p, d, o, res, st, kt);
    // BF16-stored F until close to the target (or stalled), then FP32 polish iterations.
    PhaseRule rule;
    rule.handoff = o->stop_mode == MCF_STOP_NONE ? 0.0 : 10.0 * o->eps;
    rule.stall_checks = o->stop_mode == MCF_STOP_NONE ? 0 : 5;
    rule.skip_outputs = true;
    int rc = solve_t<float, __nv_bfloat16>(p, d, o, res, st, kt, rule);
    if (rc != MCF_OK && rc != MCF_ERR_NOT_CONVERGED) return rc;
    if (rc == MCF_OK && o->stop_mode != MCF_STOP_NONE) {
      if (res->T || res->Y || res->F) return device_copy_outputs(p, res);
      return rc;
    }
    const int64_t iters_bf16 = res->iters;
    rc = transfer_to_fp32(p, o, st);
    if (rc != MCF_OK) return rc;
    mcf_options o2 = *o;
    o2.precision = MCF_FP32;
    o2.warm_start = 1;
    o2.max_iters = o->polish_iters;
    mcf_kernel_times kt2{};
    cudaStream_t st2 = user ? user : p->ds->own_stream;   // the BF16 state's stream is gone
    rc = solve_t<float, float>(p, p->ds, &o2, res, st2, kt ? &kt2 : nullptr);
    if (kt)
      for (int i = 0; i < 4; ++i) { kt->ms[i] += kt2.ms[i]; kt->launches[i] += kt2.launches[i]; }
    if (kt) kt->ms_total += kt2.ms_total;
    res->iters += iters_bf16;
    return rc;
  }
  return solve_t<float, float>(p, d, o, res, st, kt);
}

}  // namespace pdmcf
