// pdmcf_internal.h — host-side problem record shared by the C ABI and the CUDA driver.
#pragma once

#include <stdint.h>

#include <atomic>
#include <memory>
#include <mutex>
#include <algorithm>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "pdmcf.h"

namespace pdmcf {
struct DeviceState;   // defined in pdmcf_solver.cu

void set_error(const std::string& msg);   // thread-local message for mcf_last_error()
// Unique id of the calling thread's current CUDA context, 0 if none (pdmcf_noalloc.cu).
unsigned long long current_context_id();

// Internal edge order: edges sorted by head, so each node's in-edges are one contiguous
// range of rows of F; out-edges are listed through out_ptr/out_idx.
struct Topology {
  std::vector<int32_t> perm;     // internal edge e -> caller's edge index
  std::vector<int32_t> e_tail, e_head;
  std::vector<int32_t> in_ptr;   // n+1
  std::vector<int32_t> out_ptr;  // n+1
  std::vector<int32_t> out_idx;  // m internal edge ids, grouped by tail
  int dmax = 0;                  // max in+out degree (Appendix A)
  // Node renumbering: caller node -> internal node (empty = identity). A relabelling of the
  // nodes leaves the problem unchanged; e_tail/e_head, in_ptr/out_ptr and every device row
  // and column use internal numbers, and inputs/outputs are mapped at the boundary.
  std::vector<int32_t> node_of;
  int node(int caller) const { return node_of.empty() ? caller : node_of[caller]; }
};

// Allocator whose value-less construct() leaves doubles uninitialised, so resizing a host
// copy of an n x n matrix does not write (and page in) every page on one thread before the
// parallel copy does.
template <typename T>
struct DefaultInitAlloc : std::allocator<T> {
  template <typename U> struct rebind { using other = DefaultInitAlloc<U>; };
  DefaultInitAlloc() = default;
  template <typename U> DefaultInitAlloc(const DefaultInitAlloc<U>&) noexcept {}
  template <typename U> void construct(U* q) noexcept { ::new ((void*)q) U; }
  template <typename U, typename... A> void construct(U* q, A&&... a) {
    ::new ((void*)q) U(std::forward<A>(a)...);
  }
};
using HostMatrix = std::vector<double, DefaultInitAlloc<double>>;

// Runs fn(u0, u1) over ranges of [0, units) on up to 16 host threads when the work covers
// at least 32 MB (unit_bytes per unit), else on the calling thread. Host passes over n x n
// matrices (validation, copies, the first touch of fresh pages) scale with the cores; a
// range whose thread cannot be started runs on the calling thread.
template <typename Fn>
inline void parallel_ranges(int64_t units, size_t unit_bytes, Fn fn) {
  int64_t nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  if ((double)units * (double)unit_bytes < (double)(32u << 20)) nt = 1;
  nt = std::min<int64_t>(nt, std::max<int64_t>(units, 1));
  std::vector<std::thread> th;
  for (int64_t k = 1; k < nt; ++k) {
    const int64_t u0 = units * k / nt, u1 = units * (k + 1) / nt;
    try {
      th.emplace_back(fn, u0, u1);
    } catch (...) {
      fn(u0, u1);
    }
  }
  fn((int64_t)0, units / nt);
  for (auto& t : th) t.join();
}

// Writes one zero per 4 KB into [p, p + bytes) on parallel threads, so that a fresh output
// buffer's pages are mapped (and zeroed by the system) in parallel rather than during a
// single-threaded device-to-host copy. The contents are then overwritten.
inline void prefault_host(void* p, size_t bytes) {
  if (!p || bytes == 0) return;
  constexpr size_t kPage = 4096;
  unsigned char* b = static_cast<unsigned char*>(p);
  parallel_ranges((int64_t)((bytes + kPage - 1) / kPage), kPage, [b, bytes](int64_t q0, int64_t q1) {
    for (int64_t q = q0; q < q1; ++q) {
      const size_t off = (size_t)q * kPage;
      if (off < bytes) reinterpret_cast<volatile unsigned char*>(b)[off] = 0;
    }
  });
}

}  // namespace pdmcf

struct mcf_problem {
  int32_t n = 0, m = 0;
  int kind = MCF_LOG;
  std::vector<int32_t> tail, head;     // caller order
  std::vector<double> cap;             // caller order
  pdmcf::HostMatrix w;                 // n*n, w[i*n+j]
  double gamma_scalar = 0.5;
  pdmcf::HostMatrix gamma_mat;         // n*n or empty
  pdmcf::Topology topo;
  double eta = 0.0;
  double omega = 1.0;                  // resident primal weight (warm start)
  bool data_dirty = true;              // cap / w changed since the last upload
  pdmcf::DeviceState* ds = nullptr;
  std::mutex lock;                     // one call at a time per problem
  std::atomic<int> busy{0};            // >0 while a ticket uses the problem
};

namespace pdmcf {
int validate_options(const mcf_options* o);   // pdmcf_capi.cpp
// Implemented in pdmcf_solver.cu.
int device_solve(mcf_problem* p, const mcf_options* o, mcf_result* res,
                 mcf_kernel_times* kt = nullptr);
int device_copy_outputs(mcf_problem* p, mcf_result* res);
int device_save_state(mcf_problem* p, const char* path);
int device_load_state(mcf_problem* p, const char* path, int device);
void device_free(mcf_problem* p);
int64_t device_bytes(const mcf_problem* p, int precision);
}  // namespace pdmcf
