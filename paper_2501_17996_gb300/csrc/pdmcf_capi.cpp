// pdmcf_capi.cpp — the extern "C" boundary of libpdmcf.so (declared in include/pdmcf.h).
//
// Validates the problem data of Eq. (e-prob) (Zhang & Boyd, Sec. 1.1), builds the internal
// edge order, and forwards solves to the CUDA driver (pdmcf_solver.cu) and the serving
// scheduler (pdmcf_serve.cpp). No numerical work happens here.
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <limits>
#include <numeric>
#include <string>
#include <vector>

#include "pdmcf_internal.h"

namespace pdmcf {

int mcf_shape_count();

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

// A ticket of the problem has not been collected yet (see mcf_submit).
static const char* const kOutstanding =
    "the problem has an outstanding ticket (collect it with mcf_poll or mcf_wait, or discard "
    "it with mcf_cancel)";

static int fail(int code, const std::string& msg) {
  set_error(msg);
  return code;
}

// Strong connectivity (Sec. 1.1: a directed path between every pair): every node is
// reachable from node 0 along edges and along reversed edges.
static bool strongly_connected(int n, const std::vector<int32_t>& tail,
                               const std::vector<int32_t>& head) {
  for (int dir = 0; dir < 2; ++dir) {
    std::vector<std::vector<int32_t>> adj(n);
    for (size_t l = 0; l < tail.size(); ++l) {
      if (dir == 0) adj[tail[l]].push_back(head[l]);
      else adj[head[l]].push_back(tail[l]);
    }
    std::vector<char> seen(n, 0);
    std::vector<int32_t> stack{0};
    seen[0] = 1;
    int count = 1;
    while (!stack.empty()) {
      const int v = stack.back();
      stack.pop_back();
      for (int u : adj[v])
        if (!seen[u]) { seen[u] = 1; ++count; stack.push_back(u); }
    }
    if (count != n) return false;
  }
  return true;
}

// Reverse Cuthill-McKee order of the undirected version of the network: breadth-first from
// a pseudo-peripheral node (the farthest, lowest-degree node of a breadth-first sweep, twice),
// neighbours visited by increasing degree, then reversed. On networks with geometric locality
// (the k-nearest-neighbour graphs of Sec. 3.1) it puts the two ends of most edges at nearby
// numbers, so the edge phase's Y-row gathers for consecutive edges hit the same L2 lines.
static std::vector<int32_t> rcm_order(int n, const std::vector<int32_t>& tail,
                                      const std::vector<int32_t>& head) {
  std::vector<std::vector<int32_t>> adj(n);
  for (size_t e = 0; e < tail.size(); ++e) {
    adj[tail[e]].push_back(head[e]);
    adj[head[e]].push_back(tail[e]);
  }
  for (auto& a : adj) {
    std::sort(a.begin(), a.end());
    a.erase(std::unique(a.begin(), a.end()), a.end());
  }
  auto deg = [&](int v) { return (int)adj[v].size(); };
  for (auto& a : adj)
    std::stable_sort(a.begin(), a.end(), [&](int x, int y) { return deg(x) < deg(y); });
  std::vector<int32_t> order;
  std::vector<int32_t> level(n);
  auto bfs = [&](int s) {   // fills `order` (Cuthill-McKee order from s) and `level`
    order.clear();
    std::fill(level.begin(), level.end(), -1);
    level[s] = 0;
    order.push_back(s);
    for (size_t q = 0; q < order.size(); ++q)
      for (int u : adj[order[q]])
        if (level[u] < 0) { level[u] = level[order[q]] + 1; order.push_back(u); }
  };
  int start = 0;
  for (int v = 1; v < n; ++v)
    if (deg(v) < deg(start)) start = v;
  for (int sweep = 0; sweep < 2; ++sweep) {
    bfs(start);
    const int last = level[order.back()];
    int best = order.back();
    for (int v : order)
      if (level[v] == last && deg(v) < deg(best)) best = v;
    start = best;
  }
  bfs(start);
  std::reverse(order.begin(), order.end());
  return order;   // the network is connected, so every node appears once
}

static void build_topology(int n, const std::vector<int32_t>& tail_in,
                           const std::vector<int32_t>& head_in, Topology& t) {
  const int m = (int)tail_in.size();
  // renumber the nodes when that shortens the mean edge span |tail - head| at least 4x
  t.node_of.clear();
  {
    const std::vector<int32_t> order = rcm_order(n, tail_in, head_in);
    std::vector<int32_t> pos(n);
    for (int k = 0; k < n; ++k) pos[order[k]] = k;
    double span0 = 0.0, span1 = 0.0;
    for (int e = 0; e < m; ++e) {
      span0 += std::abs((double)tail_in[e] - head_in[e]);
      span1 += std::abs((double)pos[tail_in[e]] - pos[head_in[e]]);
    }
    if (4.0 * span1 <= span0) t.node_of = pos;
  }
  std::vector<int32_t> tail(m), head(m);
  for (int e = 0; e < m; ++e) {
    tail[e] = t.node(tail_in[e]);
    head[e] = t.node(head_in[e]);
  }
  t.perm.resize(m);
  std::iota(t.perm.begin(), t.perm.end(), 0);
  std::stable_sort(t.perm.begin(), t.perm.end(),
                   [&](int a, int b) { return head[a] < head[b]; });
  t.e_tail.resize(m);
  t.e_head.resize(m);
  for (int e = 0; e < m; ++e) {
    t.e_tail[e] = tail[t.perm[e]];
    t.e_head[e] = head[t.perm[e]];
  }
  t.in_ptr.assign(n + 1, 0);
  t.out_ptr.assign(n + 1, 0);
  for (int e = 0; e < m; ++e) {
    t.in_ptr[t.e_head[e] + 1]++;
    t.out_ptr[t.e_tail[e] + 1]++;
  }
  for (int j = 0; j < n; ++j) {
    t.in_ptr[j + 1] += t.in_ptr[j];
    t.out_ptr[j + 1] += t.out_ptr[j];
  }
  t.out_idx.resize(m);
  std::vector<int32_t> fill(t.out_ptr.begin(), t.out_ptr.end() - 1);
  for (int e = 0; e < m; ++e) t.out_idx[fill[t.e_tail[e]]++] = e;
  t.dmax = 0;
  for (int j = 0; j < n; ++j) {
    const int d = (t.in_ptr[j + 1] - t.in_ptr[j]) + (t.out_ptr[j + 1] - t.out_ptr[j]);
    t.dmax = std::max(t.dmax, d);
  }
}

// Copies the n x n matrix src into dst, checking ok(x) on every off-diagonal entry; on a
// failing entry returns MCF_ERR_INVALID with msg (dst is then unspecified).
template <typename Ok>
static int copy_matrix(int n, const double* src, pdmcf::HostMatrix& dst, Ok ok, const char* msg) {
  dst.resize((size_t)n * n);
  std::atomic<bool> bad{false};
  double* out = dst.data();
  pdmcf::parallel_ranges(n, (size_t)n * sizeof(double), [&](int64_t r0, int64_t r1) {
    for (int i = (int)r0; i < (int)r1; ++i) {
      const double* a = src + (size_t)i * n;
      double* b = out + (size_t)i * n;
      bool rok = true;
      for (int j = 0; j < n; ++j) {
        const double x = a[j];
        b[j] = x;
        if (j != i && !ok(x)) rok = false;
      }
      if (!rok) { bad.store(true, std::memory_order_relaxed); return; }
    }
  });
  return bad.load() ? fail(MCF_ERR_INVALID, msg) : MCF_OK;
}

static int copy_weights(int n, const double* w, pdmcf::HostMatrix& dst) {
  if (!w) return fail(MCF_ERR_INVALID, "w is NULL");
  return copy_matrix(n, w, dst, [](double x) { return x > 0.0 && std::isfinite(x); },
                     "weights must be finite and > 0 off the diagonal");
}

static int check_caps(int m, const double* cap) {
  if (!cap) return fail(MCF_ERR_INVALID, "cap is NULL");
  for (int l = 0; l < m; ++l)
    if (!(cap[l] > 0.0) || !std::isfinite(cap[l]))
      return fail(MCF_ERR_INVALID, "capacities must be finite and > 0");
  return MCF_OK;
}

int validate_options(const mcf_options* o) {
  if (!o) return fail(MCF_ERR_INVALID, "options are NULL");
  if (o->stop_mode != MCF_STOP_PAPER && o->stop_mode != MCF_STOP_REL_KKT &&
      o->stop_mode != MCF_STOP_NONE)
    return fail(MCF_ERR_INVALID, "unknown stop_mode");
  if (o->stop_mode != MCF_STOP_NONE && !(o->eps > 0.0))
    return fail(MCF_ERR_INVALID, "eps must be > 0");
  if (o->max_iters < 1) return fail(MCF_ERR_INVALID, "max_iters must be >= 1");
  if (!(o->rho > 0.0 && o->rho < 2.0)) return fail(MCF_ERR_INVALID, "rho must be in (0, 2)");
  if (!(o->theta >= 0.0 && o->theta <= 1.0)) return fail(MCF_ERR_INVALID, "theta must be in [0, 1]");
  if (o->k_adapt < 1) return fail(MCF_ERR_INVALID, "k_adapt must be >= 1");
  if (o->k_check < 1) return fail(MCF_ERR_INVALID, "k_check must be >= 1");
  if (o->precision != MCF_FP32 && o->precision != MCF_FP64 && o->precision != MCF_BF16_F)
    return fail(MCF_ERR_INVALID, "unknown precision");
  if (o->polish_iters < 0) return fail(MCF_ERR_INVALID, "polish_iters must be >= 0");
  if (o->stall_checks < 0) return fail(MCF_ERR_INVALID, "stall_checks must be >= 0");
  if (o->shape < -1 || o->shape >= mcf_shape_count()) return fail(MCF_ERR_INVALID, "unknown shape");
  if (!(o->adapt_guard >= 0.0) || !std::isfinite(o->adapt_guard))
    return fail(MCF_ERR_INVALID, "adapt_guard must be finite and >= 0");
  if (!(o->adapt_guard_below > 0.0))
    return fail(MCF_ERR_INVALID, "adapt_guard_below must be > 0");
  return MCF_OK;
}

}  // namespace pdmcf

using namespace pdmcf;

extern "C" {

const char* mcf_last_error(void) { return g_last_error.c_str(); }

const char* mcf_version(void) { return "pdmcf-gb300 0.1 (sm_103a)"; }

void mcf_options_default(mcf_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->eps = 1e-4;
  o->stop_mode = MCF_STOP_REL_KKT;
  o->max_iters = 100000;
  o->rho = 1.9;          // Sec. 2.2
  o->theta = 0.5;        // Sec. 2.4
  o->k_adapt = 100;      // Sec. 2.4
  o->tau = 1e-5;         // Sec. 2.4, Algorithm 2.1 step 3
  o->omega_freeze_iter = -1;
  o->k_check = 50;
  o->precision = MCF_FP32;
  o->warm_start = 0;
  o->polish_iters = 0;
  o->use_graphs = 1;
  o->device = 0;
  o->cuda_stream = nullptr;
  o->omega0 = 1.0;       // Sec. 2.5
  o->stall_checks = 100;
  o->compensated_duals = 1;
  o->autotune = 1;
  o->shape = -1;
  o->adapt_guard = 10.0;
  o->adapt_guard_below = 1e-2;
}

int mcf_create_problem(int32_t n, int32_t m, const int32_t* tail, const int32_t* head,
                       const double* cap, int utility_kind, const double* w,
                       const double* gamma, int64_t gamma_len, mcf_problem** out) {
  if (!out) return fail(MCF_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (n < 2) return fail(MCF_ERR_INVALID, "n must be >= 2");
  if (m < 1) return fail(MCF_ERR_INVALID, "m must be >= 1");
  if (!tail || !head) return fail(MCF_ERR_INVALID, "tail/head are NULL");
  if (utility_kind != MCF_LOG && utility_kind != MCF_POW)
    return fail(MCF_ERR_INVALID, "utility_kind must be MCF_LOG or MCF_POW");
  if ((int64_t)n * (int64_t)n > (int64_t)1 << 40) return fail(MCF_ERR_INVALID, "n too large");
  std::vector<int32_t> t(tail, tail + m), h(head, head + m);
  std::vector<int64_t> keys(m);
  for (int l = 0; l < m; ++l) {
    if (t[l] < 0 || t[l] >= n || h[l] < 0 || h[l] >= n)
      return fail(MCF_ERR_INVALID, "edge endpoint out of range");
    if (t[l] == h[l]) return fail(MCF_ERR_INVALID, "self loops are not allowed");
    keys[l] = (int64_t)t[l] * n + h[l];
  }
  std::sort(keys.begin(), keys.end());
  if (std::adjacent_find(keys.begin(), keys.end()) != keys.end())
    return fail(MCF_ERR_INVALID, "duplicate (tail, head) edge");
  int rc = check_caps(m, cap);
  if (rc != MCF_OK) return rc;
  pdmcf::HostMatrix wcopy;
  rc = copy_weights(n, w, wcopy);
  if (rc != MCF_OK) return rc;
  double gscalar = 0.5;
  pdmcf::HostMatrix gmat;
  if (utility_kind == MCF_POW) {
    if (!gamma || (gamma_len != 1 && gamma_len != (int64_t)n * n))
      return fail(MCF_ERR_INVALID, "power utility needs gamma of length 1 or n*n");
    if (gamma_len == 1) {
      gscalar = gamma[0];
      if (!(gscalar > 0.0 && gscalar < 1.0)) return fail(MCF_ERR_INVALID, "gamma must be in (0, 1)");
    } else {
      rc = copy_matrix(n, gamma, gmat, [](double x) { return x > 0.0 && x < 1.0; },
                       "gamma must be in (0, 1)");
      if (rc != MCF_OK) return rc;
    }
  }
  if (!strongly_connected(n, t, h))
    return fail(MCF_ERR_NOT_CONNECTED, "network is not strongly connected");
  mcf_problem* p = new mcf_problem();
  p->n = n;
  p->m = m;
  p->kind = utility_kind;
  p->tail = std::move(t);
  p->head = std::move(h);
  p->cap.assign(cap, cap + m);
  p->w = std::move(wcopy);
  p->gamma_scalar = gscalar;
  p->gamma_mat = std::move(gmat);
  build_topology(n, p->tail, p->head, p->topo);
  p->eta = 1.0 / std::sqrt(2.0 * (double)p->topo.dmax);   // Eq. (e-eta)
  *out = p;
  return MCF_OK;
}

int mcf_update_capacities(mcf_problem* p, const double* cap) {
  if (!p) return fail(MCF_ERR_INVALID, "problem is NULL");
  if (p->busy.load() > 0) return fail(MCF_ERR_BUSY, kOutstanding);
  int rc = check_caps(p->m, cap);
  if (rc != MCF_OK) return rc;
  std::lock_guard<std::mutex> g(p->lock);
  p->cap.assign(cap, cap + p->m);
  p->data_dirty = true;
  return MCF_OK;
}

int mcf_update_weights(mcf_problem* p, const double* w) {
  if (!p) return fail(MCF_ERR_INVALID, "problem is NULL");
  if (p->busy.load() > 0) return fail(MCF_ERR_BUSY, kOutstanding);
  pdmcf::HostMatrix wcopy;
  int rc = copy_weights(p->n, w, wcopy);
  if (rc != MCF_OK) return rc;
  std::lock_guard<std::mutex> g(p->lock);
  p->w.swap(wcopy);
  p->data_dirty = true;
  return MCF_OK;
}

int mcf_destroy_problem(mcf_problem* p) {
  if (!p) return MCF_OK;
  if (p->busy.load() > 0) return fail(MCF_ERR_BUSY, kOutstanding);
  {
    std::lock_guard<std::mutex> g(p->lock);
    device_free(p);
  }
  delete p;
  return MCF_OK;
}

int mcf_problem_size(const mcf_problem* p, int32_t* n, int32_t* m) {
  if (!p) return fail(MCF_ERR_INVALID, "problem is NULL");
  if (n) *n = p->n;
  if (m) *m = p->m;
  return MCF_OK;
}

int mcf_problem_node_order(const mcf_problem* p, int32_t* node_of) {
  if (!p) return fail(MCF_ERR_INVALID, "problem is NULL");
  if (node_of)
    for (int i = 0; i < p->n; ++i) node_of[i] = p->topo.node(i);
  return p->topo.node_of.empty() ? 0 : 1;
}

int mcf_problem_edge_order(const mcf_problem* p, int32_t* edge_of) {
  if (!p || !edge_of) return fail(MCF_ERR_INVALID, "problem or edge_of is NULL");
  for (int e = 0; e < p->m; ++e) edge_of[e] = p->topo.perm[e];
  return MCF_OK;
}

int64_t mcf_problem_device_bytes(const mcf_problem* p, int precision) {
  if (!p) return fail(MCF_ERR_INVALID, "problem is NULL");
  return device_bytes(p, precision);
}

static int solve_common(mcf_problem* p, const mcf_options* opts, mcf_result* res,
                        mcf_kernel_times* kt) {
  if (!p || !res) return fail(MCF_ERR_INVALID, "problem or result is NULL");
  if (p->busy.load() > 0) return fail(MCF_ERR_BUSY, kOutstanding);
  int rc = validate_options(opts);
  if (rc != MCF_OK) return rc;
  const auto t0 = std::chrono::steady_clock::now();
  std::lock_guard<std::mutex> g(p->lock);
  rc = device_solve(p, opts, res, kt);
  res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (rc == MCF_OK || rc == MCF_ERR_NOT_CONVERGED || rc == MCF_ERR_NUMERIC) res->status = rc;
  return rc;
}

int mcf_autotune(mcf_problem* p, const mcf_options* opts, int* best_shape, double* ms_per_iter) {
  if (!p || !best_shape) return fail(MCF_ERR_INVALID, "problem or best_shape is NULL");
  if (p->busy.load() > 0) return fail(MCF_ERR_BUSY, kOutstanding);
  int rc = validate_options(opts);
  if (rc != MCF_OK) return rc;
  std::lock_guard<std::mutex> g(p->lock);
  const int vw = opts->precision == MCF_FP64 ? 2 : (opts->precision == MCF_BF16_F ? 8 : 4);
  const int nchunks = ((p->n + 7) / 8 * 8) / vw;
  int group[64], vpt[64], pipelined[64];
  const int count = mcf_shape_info(group, vpt, nullptr, pipelined);
  int cap0 = 0;
  for (int s = 0; s < count; ++s)
    if (!pipelined[s] && group[s] * vpt[s] >= nchunks && (cap0 == 0 || group[s] * vpt[s] < cap0))
      cap0 = group[s] * vpt[s];
  int best = -1;
  double best_ms = 1e300;
  const int nchunks_rows = ((p->n + 7) / 8 * 8) / 4;   // kinds 1 and 2: 4-entry chunks
  for (int s = 0; s < count; ++s) {
    const int cap = group[s] * vpt[s];
    if (cap < (pipelined[s] ? nchunks_rows : nchunks)) continue;
    if (pipelined[s] ? opts->precision == MCF_FP64 : cap > 4 * cap0) continue;
    mcf_options o = *opts;
    o.shape = s;
    o.stop_mode = MCF_STOP_NONE;
    o.warm_start = 0;
    o.max_iters = 3;
    mcf_result r{};
    if (device_solve(p, &o, &r) != MCF_OK) continue;
    o.warm_start = 1;
    o.max_iters = 10;
    o.k_check = 10;
    mcf_kernel_times kt{};
    if (device_solve(p, &o, &r, &kt) != MCF_OK) continue;
    const double ms = kt.ms_total / 10.0;
    if (ms < best_ms) { best_ms = ms; best = s; }
  }
  device_free(p);   // tuning iterates are not a resident solution
  if (best < 0) return fail(MCF_ERR_INVALID, "no launch shape ran for this problem");
  *best_shape = best;
  if (ms_per_iter) *ms_per_iter = best_ms;
  return MCF_OK;
}

int mcf_save_state(mcf_problem* p, const char* path) {
  if (!p || !path) return fail(MCF_ERR_INVALID, "problem or path is NULL");
  if (p->busy.load() > 0) return fail(MCF_ERR_BUSY, kOutstanding);
  std::lock_guard<std::mutex> g(p->lock);
  return device_save_state(p, path);
}

int mcf_load_state(mcf_problem* p, const char* path, int device) {
  if (!p || !path) return fail(MCF_ERR_INVALID, "problem or path is NULL");
  if (p->busy.load() > 0) return fail(MCF_ERR_BUSY, kOutstanding);
  std::lock_guard<std::mutex> g(p->lock);
  return device_load_state(p, path, device);
}

int mcf_solve(mcf_problem* p, const mcf_options* opts, mcf_result* res) {
  return solve_common(p, opts, res, nullptr);
}

int mcf_solve_timed(mcf_problem* p, const mcf_options* opts, mcf_result* res,
                    mcf_kernel_times* kt) {
  if (!kt) return fail(MCF_ERR_INVALID, "kernel times pointer is NULL");
  return solve_common(p, opts, res, kt);
}

}  // extern "C"
