// pdmcf_batch.cu — BatchEngine: many resident instances advanced together, and the
// synchronous batched solve mcf_solve_batch.
//
// Per iteration: for every non-empty shape class one edge, one node and one check launch
// over the class's work list, then one scalar launch with a block per instance. Instance
// scalars live on the device (BatchScalars), so a chunk of iterations is captured once as a
// CUDA graph and replayed whatever the mix; the host reads the scalar mirror once per chunk
// to retire finished instances and admit new ones between chunks.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "pdmcf_batch_engine.h"

namespace pdmcf {

// Solver-side helpers (pdmcf_solver.cu).
int batch_prepare_state(mcf_problem* p, const mcf_options* o, cudaStream_t st, bool* warm);
void batch_state_pointers(mcf_problem* p, BatchInst* bi, int* parity);
void batch_finish_state(mcf_problem* p, int parity, const DevScalars& s, cudaStream_t st);

// ------------------------------------------------------------------ scalar kernel

struct BatchScalarArgs {
  const BatchInst* insts;
  const int* slots;
  const int* nslots;
};

// One block per resident instance: fixed-order FP64 sums of its per-edge and per-node
// parts, the shared scalar update, parity flip and the stop rule (Algorithm 2.1, step 1,
// evaluated on the instance's own check iterations).
__global__ void __launch_bounds__(256) batch_scalar_kernel(BatchScalarArgs a) {
  __shared__ double sh[256];
  if ((int)blockIdx.x >= *a.nslots) return;
  const BatchInst& I = a.insts[a.slots[blockIdx.x]];
  BatchScalars* bs = I.sc;
  if (!bs->active) return;
  const bool check = batch_is_check(bs);
  const double dF2 = det_sum(I.pe, I.m, 1, 0, sh);
  const double dY2 = det_sum(I.pn, I.n, NODE_PARTS, 0, sh);
  double nodep[NODE_PARTS];
  double chk[CHECK_PARTS];
  if (check) {
    for (int f = 1; f < NODE_PARTS; ++f) nodep[f] = det_sum(I.pn, I.n, NODE_PARTS, f, sh);
    for (int f = 0; f < CHECK_PARTS; ++f) chk[f] = det_sum(I.pc, I.m, CHECK_PARTS, f, sh);
  }
  if (threadIdx.x != 0) return;
  DevScalars* s = &bs->s;
  scalar_update(s, dF2, dY2, nodep, chk, check);
  bs->parity ^= 1;
  bool stop = false;
  bool stall = false;
  if (check) {
    const double nm = (double)I.n * (double)I.m;
    if (bs->stop_mode == MCF_STOP_PAPER && s->r < nm * bs->eps) stop = true;
    if (bs->stop_mode == MCF_STOP_REL_KKT && s->rel_kkt < bs->eps) stop = true;
    const int frozen = (s->freeze >= 0 && s->freeze <= s->k) ? 1 : 0;
    if (frozen != bs->stall_frozen) {   // constant omega from here on: a new phase
      bs->stall_frozen = frozen;
      bs->stall_best = INFINITY;
      bs->stall_count = 0;
    }
    if (!stop && bs->stop_mode == MCF_STOP_REL_KKT && bs->stall_checks > 0 &&
        s->rel_kkt < 100.0 * bs->eps) {
      if (s->rel_kkt < 0.95 * bs->stall_best) { bs->stall_best = s->rel_kkt; bs->stall_count = 0; }
      else if (++bs->stall_count >= bs->stall_checks) { stall = true; bs->stalled = 1; }
    }
  }
  if (s->k >= bs->max_iters || s->numeric_error || stop || stall) {
    bs->done = stop ? 1 : 2;    // 1: stop rule held, 2: iteration cap or numeric error
    bs->active = 0;
  }
}

// ------------------------------------------------------------------ engine

int batch_admit_shape(const mcf_problem* p) {
  const int ld = (p->n + 7) / 8 * 8;
  return pick_shape(ld / 4);
}

int64_t BatchEngine::extra_bytes(const mcf_problem* p) {
  return (int64_t)sizeof(double) * ((int64_t)p->m * (1 + CHECK_PARTS) + (int64_t)p->n * NODE_PARTS);
}

BatchEngine::BatchEngine(int device, int max_slots)
    : device_(device), max_slots_(max_slots), slots_(max_slots), h_insts_(max_slots) {}

BatchEngine::~BatchEngine() {
  cudaSetDevice(device_);
  for (int s = 0; s < max_slots_; ++s)
    if (slots_[s].used) release(s);
  destroy_graphs();
  void* bufs[] = {d_insts_, d_sc_, d_slot_list_, d_nslots_, d_cls_count_, d_cls_inst_,
                  d_cls_eoff_, d_cls_noff_};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (h_sc_) cudaFreeHost(h_sc_);
  if (stream_) cudaStreamDestroy(stream_);
}

#define BCK(call)                                                                       \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      set_error(std::string("CUDA error ") + cudaGetErrorString(e_) + " in " #call);    \
      return MCF_ERR_CUDA;                                                              \
    }                                                                                   \
  } while (0)

int BatchEngine::init() {
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    set_error("no CUDA device available (the solver has no CPU path)");
    return MCF_ERR_CUDA;
  }
  BCK(cudaSetDevice(device_));
  BCK(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
  BCK(cudaDeviceGetAttribute(&sms_, cudaDevAttrMultiProcessorCount, device_));
  const size_t S = max_slots_;
  BCK(cudaMalloc((void**)&d_insts_, S * sizeof(BatchInst)));
  BCK(cudaMalloc((void**)&d_sc_, S * sizeof(BatchScalars)));
  BCK(cudaMallocHost((void**)&h_sc_, S * sizeof(BatchScalars)));
  BCK(cudaMalloc((void**)&d_slot_list_, S * sizeof(int)));
  BCK(cudaMalloc((void**)&d_nslots_, sizeof(int)));
  BCK(cudaMalloc((void**)&d_cls_count_, NUM_SHAPES * sizeof(int)));
  BCK(cudaMalloc((void**)&d_cls_inst_, NUM_SHAPES * S * sizeof(int)));
  BCK(cudaMalloc((void**)&d_cls_eoff_, NUM_SHAPES * (S + 1) * sizeof(long long)));
  BCK(cudaMalloc((void**)&d_cls_noff_, NUM_SHAPES * (S + 1) * sizeof(long long)));
  std::memset(h_sc_, 0, S * sizeof(BatchScalars));
  BCK(cudaMemsetAsync(d_sc_, 0, S * sizeof(BatchScalars), stream_));
  BCK(cudaMemsetAsync(d_nslots_, 0, sizeof(int), stream_));
  BCK(cudaMemsetAsync(d_cls_count_, 0, NUM_SHAPES * sizeof(int), stream_));
  const BatchTable& T = batch_table();
  for (int c = 0; c < NUM_SHAPES; ++c) {
    BatchKernel ks[3] = {T.edge[c], T.node[c], T.check[c]};
    for (int k = 0; k < 3; ++k) {
      int occ = 0;
      BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)ks[k], kShapes[c].block, 0));
      grid_[k][c] = std::max(1, occ) * sms_;
    }
  }
  BCK(cudaStreamSynchronize(stream_));
  return MCF_OK;
}

int BatchEngine::free_slots() const {
  int f = 0;
  for (const auto& s : slots_) f += s.used ? 0 : 1;
  return f;
}

int BatchEngine::active_count() const {
  int a = 0;
  for (const auto& s : slots_) a += (s.used && !s.finished) ? 1 : 0;
  return a;
}

int BatchEngine::add(mcf_problem* p, const mcf_options& o, void* tag, int* slot_out,
                     int cls_override) {
  int s = -1;
  for (int i = 0; i < max_slots_ && s < 0; ++i)
    if (!slots_[i].used) s = i;
  if (s < 0) {
    set_error("no free batch slot");
    return MCF_ERR_BUSY;
  }
  const int nchunks = ((p->n + 7) / 8 * 8) / 4;
  int cls = cls_override >= 0 ? cls_override : batch_admit_shape(p);
  if (cls < 0 || kShapes[cls].group * kShapes[cls].vpt < nchunks) {
    set_error("instance too large for the batched kernels or shape too small");
    return MCF_ERR_INVALID;
  }
  BCK(cudaSetDevice(device_));
  bool warm = false;
  int rc = batch_prepare_state(p, &o, stream_, &warm);
  if (rc != MCF_OK) return rc;
  BatchSlot& sl = slots_[s];
  sl = BatchSlot();
  auto A = [&](double** ptr, size_t count) {
    return cudaMalloc((void**)ptr, std::max<size_t>(count, 1) * sizeof(double)) == cudaSuccess;
  };
  if (!A(&sl.pe, p->m) || !A(&sl.pn, (size_t)p->n * NODE_PARTS) ||
      !A(&sl.pc, (size_t)p->m * CHECK_PARTS)) {
    cudaGetLastError();
    for (double* b : {sl.pe, sl.pn, sl.pc})
      if (b) cudaFree(b);
    sl = BatchSlot();
    set_error("device allocation failed");
    return MCF_ERR_OOM;
  }
  BCK(cudaMemsetAsync(sl.pc, 0, (size_t)p->m * CHECK_PARTS * sizeof(double), stream_));
  BCK(cudaMemsetAsync(sl.pn, 0, (size_t)p->n * NODE_PARTS * sizeof(double), stream_));
  sl.used = true;
  sl.p = p;
  sl.opts = o;
  sl.tag = tag;
  sl.cls = cls;
  sl.bytes = device_bytes(p, MCF_FP32) + extra_bytes(p);
  BatchInst bi{};
  int parity0 = 0;
  batch_state_pointers(p, &bi, &parity0);
  bi.rho = (float)o.rho;
  bi.pe = sl.pe;
  bi.pn = sl.pn;
  bi.pc = sl.pc;
  bi.sc = d_sc_ + s;
  h_insts_[s] = bi;
  BatchScalars& hs = h_sc_[s];
  std::memset(&hs, 0, sizeof(hs));
  DevScalars& d = hs.s;
  d.eta = p->eta;
  d.omega = p->omega;
  d.alpha = d.eta / d.omega;
  d.beta = d.eta * d.omega;
  d.alpha_last = d.alpha;
  d.beta_last = d.beta;
  d.theta = o.theta;
  d.tau = o.tau;
  d.k_adapt = o.k_adapt > 0 ? o.k_adapt : 1;
  d.freeze = o.omega_freeze_iter;
  d.guard = o.adapt_guard;
  d.guard_below = o.adapt_guard_below;
  d.omega_ref = 0.0;
  d.omega_arm = 0.0;
  d.best_kkt = INFINITY;
  d.r = INFINITY;
  d.rel_kkt = INFINITY;
  d.n = p->n;
  d.m = p->m;
  hs.parity = parity0;
  hs.active = 1;
  hs.done = 0;
  hs.stop_mode = o.stop_mode;
  hs.max_iters = o.max_iters;
  hs.k_check = std::max(1, o.k_check);
  hs.eps = o.eps;
  hs.stall_checks = o.stall_checks;
  hs.stall_best = INFINITY;
  hs.stall_frozen = 0;
  BCK(cudaMemcpyAsync(d_insts_ + s, &bi, sizeof(bi), cudaMemcpyHostToDevice, stream_));
  BCK(cudaMemcpyAsync(d_sc_ + s, &hs, sizeof(hs), cudaMemcpyHostToDevice, stream_));
  BCK(cudaStreamSynchronize(stream_));
  (void)warm;
  lists_dirty_ = true;
  *slot_out = s;
  return MCF_OK;
}

// Class work lists (slot order within a class) and the scalar kernel's slot list.
int BatchEngine::upload_lists() {
  const size_t S = max_slots_;
  std::vector<int> count(NUM_SHAPES, 0), inst(NUM_SHAPES * S, 0), slot_list;
  std::vector<long long> eoff(NUM_SHAPES * (S + 1), 0), noff(NUM_SHAPES * (S + 1), 0);
  unsigned mask = 0;
  for (int s = 0; s < max_slots_; ++s) {
    const BatchSlot& sl = slots_[s];
    if (!sl.used || sl.finished) continue;
    const int c = sl.cls;
    const int k = count[c]++;
    inst[c * S + k] = s;
    eoff[c * (S + 1) + k + 1] = eoff[c * (S + 1) + k] + sl.p->m;
    noff[c * (S + 1) + k + 1] = noff[c * (S + 1) + k] + sl.p->n;
    slot_list.push_back(s);
    mask |= 1u << c;
  }
  const int ns = (int)slot_list.size();
  if (slot_list.empty()) slot_list.push_back(0);
  BCK(cudaMemcpyAsync(d_cls_count_, count.data(), NUM_SHAPES * sizeof(int), cudaMemcpyHostToDevice, stream_));
  BCK(cudaMemcpyAsync(d_cls_inst_, inst.data(), inst.size() * sizeof(int), cudaMemcpyHostToDevice, stream_));
  BCK(cudaMemcpyAsync(d_cls_eoff_, eoff.data(), eoff.size() * sizeof(long long), cudaMemcpyHostToDevice, stream_));
  BCK(cudaMemcpyAsync(d_cls_noff_, noff.data(), noff.size() * sizeof(long long), cudaMemcpyHostToDevice, stream_));
  BCK(cudaMemcpyAsync(d_slot_list_, slot_list.data(), slot_list.size() * sizeof(int), cudaMemcpyHostToDevice, stream_));
  BCK(cudaMemcpyAsync(d_nslots_, &ns, sizeof(int), cudaMemcpyHostToDevice, stream_));
  BCK(cudaStreamSynchronize(stream_));   // host staging vectors die at return
  class_mask_ = mask;
  lists_dirty_ = false;
  return MCF_OK;
}

int BatchEngine::launch_iteration(cudaStream_t st, bool with_check) {
  const BatchTable& T = batch_table();
  const size_t S = max_slots_;
  for (int c = 0; c < NUM_SHAPES; ++c) {
    if (!(class_mask_ & (1u << c))) continue;
    BatchClassDev cls{d_cls_count_ + c, d_cls_inst_ + c * S, d_cls_eoff_ + c * (S + 1),
                      d_cls_noff_ + c * (S + 1)};
    const BatchInst* insts = d_insts_;
    void* kargs[] = {(void*)&insts, &cls};
    const int block = kShapes[c].block;
    BCK(cudaLaunchKernel((const void*)T.edge[c], dim3(grid_[0][c]), dim3(block), kargs, 0, st));
    BCK(cudaLaunchKernel((const void*)T.node[c], dim3(grid_[1][c]), dim3(block), kargs, 0, st));
    if (with_check)
      BCK(cudaLaunchKernel((const void*)T.check[c], dim3(grid_[2][c]), dim3(block), kargs, 0, st));
  }
  BatchScalarArgs sa{d_insts_, d_slot_list_, d_nslots_};
  batch_scalar_kernel<<<max_slots_, 256, 0, st>>>(sa);
  BCK(cudaGetLastError());
  return MCF_OK;
}

void BatchEngine::destroy_graphs() {
  for (auto& kv : graphs_) cudaGraphExecDestroy(kv.second);
  graphs_.clear();
}

int BatchEngine::step(int iters) {
  nvtxRangePushA("pdmcf batched chunk");
  const int rc = step_impl(iters);
  nvtxRangePop();
  return rc;
}

// Iterations i of the next chunk (bit i) in which some active instance takes a stop test
// (batch_is_check at its k = k0 + i): the check launch of the other iterations would find
// nothing to do for any instance, so it is left out. Chunks longer than 64 iterations keep it
// in every iteration.
uint64_t BatchEngine::check_iterations(int iters) const {
  if (iters > 64) return ~0ull;
  uint64_t mask = 0;
  for (int s = 0; s < max_slots_; ++s) {
    const BatchSlot& sl = slots_[s];
    const BatchScalars& h = h_sc_[s];
    if (!sl.used || sl.finished || !h.active) continue;
    const long long kc = std::max(1LL, h.k_check);
    for (int i = 0; i < iters; ++i) {
      const long long k1 = h.s.k + i + 1;
      if (k1 % kc == 0 || k1 >= h.max_iters) mask |= 1ull << i;
    }
  }
  return mask;
}

int BatchEngine::step_impl(int iters) {
  BCK(cudaSetDevice(device_));
  if (lists_dirty_) {
    int rc = upload_lists();
    if (rc != MCF_OK) return rc;
  }
  if (class_mask_ == 0) return MCF_OK;
  const uint64_t checks = check_iterations(iters);
  auto with_check = [&](int i) { return i >= 64 || ((checks >> i) & 1ull) != 0; };
  const auto key = std::make_tuple(class_mask_, iters, checks);
  auto it = graphs_.find(key);
  if (it == graphs_.end() && !graphs_broken_) {
    if (graphs_.size() >= 64) destroy_graphs();   // bound the cache
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    bool ok = cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    for (int i = 0; i < iters && ok; ++i) ok = launch_iteration(stream_, with_check(i)) == MCF_OK;
    const cudaError_t e = cudaStreamEndCapture(stream_, &g);
    ok = ok && e == cudaSuccess && g && cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
      cudaGetLastError();
      graphs_broken_ = true;
    } else {
      it = graphs_.emplace(key, ge).first;
    }
  }
  if (it != graphs_.end()) {
    BCK(cudaGraphLaunch(it->second, stream_));
  } else {
    for (int i = 0; i < iters; ++i) {
      int rc = launch_iteration(stream_, with_check(i));
      if (rc != MCF_OK) return rc;
    }
  }
  BCK(cudaMemcpyAsync(h_sc_, d_sc_, (size_t)max_slots_ * sizeof(BatchScalars), cudaMemcpyDeviceToHost, stream_));
  BCK(cudaStreamSynchronize(stream_));
  for (int s = 0; s < max_slots_; ++s) {
    BatchSlot& sl = slots_[s];
    if (!sl.used || sl.finished || h_sc_[s].active) continue;
    sl.finished = true;
    const DevScalars& d = h_sc_[s].s;
    if (d.numeric_error) sl.status = MCF_ERR_NUMERIC;
    else if (h_sc_[s].done == 1 || sl.opts.stop_mode == MCF_STOP_NONE) sl.status = MCF_OK;
    else sl.status = MCF_ERR_NOT_CONVERGED;
    finished_.push_back(s);
    lists_dirty_ = true;
  }
  return MCF_OK;
}

std::vector<int> BatchEngine::take_finished() {
  std::vector<int> out;
  out.swap(finished_);
  return out;
}

void BatchEngine::release(int s) {
  BatchSlot& sl = slots_[s];
  if (!sl.used) return;
  cudaSetDevice(device_);
  const DevScalars& d = h_sc_[s].s;
  mcf_result& r = sl.res;
  r.iters = d.k;
  r.feasible = d.feasible;
  r.utility = d.P;
  r.dual_bound = d.D;
  r.r = d.r;
  r.r_over_nm = d.r / ((double)sl.p->n * (double)sl.p->m);
  r.rel_gap = d.rel_gap;
  r.rel_cons = d.rel_cons;
  r.rel_stat = d.rel_stat;
  r.rel_kkt = d.rel_kkt;
  r.nonpos_frac = d.nonpos_frac;
  r.omega = d.omega;
  r.delta_f = d.dF;
  r.delta_y = d.dY;
  r.omega_frozen_at = (d.freeze >= 0 && d.freeze <= d.k) ? d.freeze : -1;
  r.stalled = h_sc_[s].stalled;
  r.status = sl.status;
  batch_finish_state(sl.p, h_sc_[s].parity, d, stream_);
  for (double* b : {sl.pe, sl.pn, sl.pc})
    if (b) cudaFree(b);
  const mcf_result keep = sl.res;
  const int st = sl.status;
  sl = BatchSlot();
  sl.res = keep;
  sl.status = st;
  h_sc_[s].active = 0;
  lists_dirty_ = true;
}

// ------------------------------------------------------------------ autotuner
// For a default class c (the smallest shape covering the chunks), the candidates are every
// shape whose capacity covers the class's largest vector and is at most 4x the class
// capacity (warp groups with more chunks per lane, or CTA groups). Each candidate runs 3 + 10
// batched iterations of 16 synthetic instances (ring plus 7 random out-edges per node, the
// class's largest n, log utility) in a private engine; the fastest per iteration wins. The
// choice depends only on the class, so an instance's shape never depends on the mix.

namespace {
std::mutex g_tune_mu;
std::map<std::pair<int, int>, int> g_tuned;   // (device, default class) -> tuned class

uint64_t splitmix(uint64_t& x) {
  uint64_t z = (x += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

mcf_problem* synthetic_problem(int n, uint64_t seed) {
  const int deg = std::min(8, n - 1);
  std::vector<int32_t> t, h;
  for (int i = 0; i < n; ++i) {
    std::vector<int32_t> used{i, (i + 1) % n};
    t.push_back(i);
    h.push_back((i + 1) % n);
    while ((int)used.size() < deg + 1) {
      const int j = (int)(splitmix(seed) % (uint64_t)n);
      if (std::find(used.begin(), used.end(), j) != used.end()) continue;
      used.push_back(j);
      t.push_back(i);
      h.push_back(j);
    }
  }
  const int m = (int)t.size();
  std::vector<double> cap(m), w((size_t)n * n, 1.0);
  for (int l = 0; l < m; ++l) cap[l] = 1.0 + 9.0 * (double)(splitmix(seed) >> 11) / 9007199254740992.0;
  for (auto& x : w) x = 0.5 + (double)(splitmix(seed) >> 11) / 9007199254740992.0;
  mcf_problem* p = nullptr;
  mcf_create_problem(n, m, t.data(), h.data(), cap.data(), MCF_LOG, w.data(), nullptr, 0, &p);
  return p;
}

int tune_class(int device, int c0) {
  const int cap0 = kShapes[c0].group * kShapes[c0].vpt;
  const int n = std::max(4, cap0 * 4 - 8);
  std::vector<int> cands;
  for (int s = 0; s < NUM_SHAPES; ++s) {
    const int cap = kShapes[s].group * kShapes[s].vpt;
    if (cap >= cap0 && cap <= 4 * cap0) cands.push_back(s);
  }
  constexpr int kCount = 16;
  std::vector<mcf_problem*> probs;
  for (int i = 0; i < kCount; ++i) probs.push_back(synthetic_problem(n, 1000003ULL * (i + 1)));
  mcf_options o;
  mcf_options_default(&o);
  o.stop_mode = MCF_STOP_NONE;
  o.max_iters = 1 << 30;
  o.device = device;
  int best = c0;
  double best_t = 1e300;
  for (int c : cands) {
    BatchEngine eng(device, kCount);
    if (eng.init() != MCF_OK) break;
    bool ok = true;
    for (int i = 0; i < kCount && ok; ++i) {
      int slot = 0;
      ok = probs[i] && eng.add(probs[i], o, nullptr, &slot, c) == MCF_OK;
    }
    if (!ok || eng.step(3) != MCF_OK) continue;
    const auto t0 = std::chrono::steady_clock::now();
    if (eng.step(10) != MCF_OK) continue;
    const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (dt < best_t) { best_t = dt; best = c; }
  }
  for (mcf_problem* p : probs) mcf_destroy_problem(p);
  return best;
}
}  // namespace

int batch_class_for(int device, int nchunks, bool autotune) {
  const int c0 = pick_shape(nchunks);
  if (c0 < 0 || !autotune) return c0;
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tuned.find({device, c0});
    if (it != g_tuned.end()) return it->second;
  }
  const int c = tune_class(device, c0);
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tuned.emplace(std::make_pair(device, c0), c);
  return g_tuned[{device, c0}];
}

}  // namespace pdmcf

using namespace pdmcf;

// Solve `count` independent problems together (FP32; one launch per phase and shape class
// for all of them). results[i] receives problem i's scalars and, if its T/F/Y pointers are
// set, its outputs. Returns MCF_OK when every problem met its stop rule.
extern "C" int mcf_solve_batch(mcf_problem** probs, int count, const mcf_options* opts,
                               mcf_result* results) {
  if (count < 0 || (count > 0 && (!probs || !results))) {
    set_error("problems or results are NULL");
    return MCF_ERR_INVALID;
  }
  int rc = pdmcf::validate_options(opts);
  if (rc != MCF_OK) return rc;
  if (opts->precision != MCF_FP32) {
    set_error("batched solves run FP32 iterates");
    return MCF_ERR_INVALID;
  }
  if (count == 0) return MCF_OK;
  for (int i = 0; i < count; ++i)
    if (probs[i] && probs[i]->busy.load() > 0) {
      set_error("a problem in the batch has an outstanding ticket (collect it with mcf_poll or "
                "mcf_wait, or discard it with mcf_cancel)");
      return MCF_ERR_BUSY;
    }
  const auto t0 = std::chrono::steady_clock::now();
  BatchEngine eng(opts->device, count);
  rc = eng.init();
  if (rc != MCF_OK) return rc;
  std::vector<std::unique_lock<std::mutex>> locks;
  for (int i = 0; i < count; ++i) {
    if (!probs[i]) {
      set_error("NULL problem in batch");
      return MCF_ERR_INVALID;
    }
    for (int j = 0; j < i; ++j)
      if (probs[j] == probs[i]) {
        set_error("a problem appears twice in the batch");
        return MCF_ERR_INVALID;
      }
    locks.emplace_back(probs[i]->lock);
    int slot = 0;
    const int nchunks = ((probs[i]->n + 7) / 8 * 8) / 4;
    const int cls = opts->shape >= 0 && opts->shape < NUM_SHAPES
                        ? opts->shape
                        : batch_class_for(opts->device, nchunks, opts->autotune != 0);
    rc = eng.add(probs[i], *opts, nullptr, &slot, cls);
    if (rc != MCF_OK) return rc;
  }
  const int chunk = std::max(1, std::min(opts->k_check, 50));
  while (eng.active_count() > 0) {
    rc = eng.step(chunk);
    if (rc != MCF_OK) return rc;
    (void)eng.take_finished();
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  int worst = MCF_OK;
  for (int i = 0; i < count; ++i) {
    eng.release(i);
    mcf_result& out = results[i];
    double *T = out.T, *F = out.F, *Y = out.Y;
    out = eng.slot(i).res;
    out.T = T;
    out.F = F;
    out.Y = Y;
    out.seconds = secs;
    if ((T || F || Y) && (out.status == MCF_OK || out.status == MCF_ERR_NOT_CONVERGED)) {
      rc = device_copy_outputs(probs[i], &out);
      if (rc != MCF_OK) return rc;
    }
    if (out.status != MCF_OK && worst == MCF_OK) worst = out.status;
  }
  return worst;
}
