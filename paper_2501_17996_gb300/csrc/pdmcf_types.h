// pdmcf_types.h — plain structs shared by the host driver and the kernels.
#pragma once

#include <stdint.h>

namespace pdmcf {

// FP64 partial sums written per block by the node and check kernels.
constexpr int NODE_PARTS = 7;   // ||dY||^2, #T<=0, sum u(T), sum (-u)^*(Y^), ||T(Y^)-T||^2, ||T||^2, #Y^>=0
constexpr int CHECK_PARTS = 4;  // ||G||^2, <G, F^-Q>, ||F^-Q||^2, sum_l c_l max(0, max_i (Y^A)_il)

// Device-resident scalar state of one solve. Kernels read alpha/beta from here, so a
// captured iteration can be replayed without host involvement.
struct DevScalars {
  // step sizes (Sec. 2.4): alpha = eta/omega, beta = eta*omega
  double eta, omega, alpha, beta;
  double alpha_last, beta_last;   // the step sizes the last completed iteration used
  long long k;           // iterations completed
  double dF, dY;         // Delta_F, Delta_Y of the last iteration (Eq. e-primal_weight)
  // primal weight rule parameters
  double theta, tau;
  long long k_adapt, freeze;
  double guard, guard_below, best_kkt, omega_ref, omega_arm;   // adaptation stop (scalar_update)
  // results of the last check iteration; check_k = k after that iteration
  long long check_k;
  double r, P, D, g_norm, rel_gap, rel_cons, rel_stat, rel_kkt, nonpos_frac;
  int feasible;
  int numeric_error;     // NaN/Inf met in a reduction
  int wait_timeout;      // a bounded device-side wait gave up (kernel returned early)
  int n, m;
};

}  // namespace pdmcf
