// pdmcf_internal.h — host-side problem record shared by the C ABI and the CUDA driver.
#pragma once

#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "pdmcf.h"

namespace pdmcf {
struct DeviceState;   // defined in pdmcf_solver.cu

void set_error(const std::string& msg);   // thread-local message for mcf_last_error()

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

}  // namespace pdmcf

struct mcf_problem {
  int32_t n = 0, m = 0;
  int kind = MCF_LOG;
  std::vector<int32_t> tail, head;     // caller order
  std::vector<double> cap;             // caller order
  std::vector<double> w;               // n*n, w[i*n+j]
  double gamma_scalar = 0.5;
  std::vector<double> gamma_mat;       // n*n or empty
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
