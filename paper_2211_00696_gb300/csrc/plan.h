// The plan object behind phikron_plan_t: everything Algorithm 6 computes before it sees v.
#pragma once

#include <vector>

#include "common.h"
#include "profile.h"

namespace phikron {

struct Plan {
  int dims = 0;
  int n[PHIKRON_MAX_DIMS] = {1, 1, 1, 1, 1, 1};
  long long N = 0;
  // sizes the mixed path computes with: n[d] rounded up to a multiple of 16 (the padded factor
  // is diag(A^d, 0), so its exponentials are diag(e^{c A^d}, I) and a zero-padded vector stays
  // zero on the pad); equal to n, N otherwise
  int pn[PHIKRON_MAX_DIMS] = {1, 1, 1, 1, 1, 1};
  long long PN = 0;
  double tau = 0.0;
  int p = 0;            // l_max: orders 0..p are returned
  double tol = 0.0;
  phikron_opts opts{};
  int s = 0, m = 0, cost = 0;
  int selector_used = 0;   // 0 Algorithm 5, 1 network, 2 network with raised m, 3 network rejected -> Algorithm 5
  double alpha = 0.0, log10_bound = 0.0;
  std::vector<double> x, w, coef;   // nodes, weights on [0,1]; coef[(j-1)*m + k]

  // unique factors: uniq_of[d] -> u, uniq_rep[u] -> first d
  int nuniq = 0;
  int uniq_of[PHIKRON_MAX_DIMS] = {0, 0, 0, 0, 0, 0};
  int uniq_rep[PHIKRON_MAX_DIMS] = {0, 0, 0, 0, 0, 0};
  // per unique factor, nexp = m + 1 + s float64 matrices n_d x n_d:
  //   [0, m)       E_k = exp((1 - x_k) 2^{-s} M^d)
  //   m            exp(M^d)                      (phi_0)
  //   m + 1 + t    G_t = exp(2^{t-s} M^d), t < s (squaring steps)
  int nexp = 0;
  double* dExp[PHIKRON_MAX_DIMS] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double* dCoef = nullptr;

  // adaptive Clenshaw-Curtis (Algorithm 2): levels 0..ad_levels with ad_nodes[l] = 6*2^l + 1
  // nodes; nodes are stored in order of first appearance, so level l uses the first
  // ad_nodes[l] exponentials; the weights of level l start at coef[ad_coef_off[l]] (p x nodes)
  int ad_levels = -1;
  std::vector<int> ad_nodes;
  std::vector<size_t> ad_coef_off;
  double* dT = nullptr;          // node vectors v_i, m x N
  unsigned long long* dErr = nullptr;  // 2p reduction slots (bit patterns of non-negative doubles)
  int last_nodes = 0;
  double last_err = 0.0;

  // the Remark's combination: [m x p] x_i^{j-1}/(j-1)!, then [m] w_i (allocated on first use)
  double* dCombo = nullptr;
  double* dY2 = nullptr;     // m vectors z_i

  // float64 apply work buffers
  double* dW1 = nullptr;
  double* dW2 = nullptr;
  double* dY = nullptr;
  double* dYn = nullptr;
  double* dV = nullptr;      // staging for phikron_apply_host
  double* dOut = nullptr;
  // second staging set, copy streams and events of phikron_apply_host_many (created by its
  // first call)
  double* dV2 = nullptr;
  double* dOut2 = nullptr;
  cudaStream_t cp_in = nullptr, cp_out = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_comp[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
  cudaEvent_t ev_start = nullptr;

  // mixed-precision state (owned by the precision back-end; see precision_setup)
  void* mixed = nullptr;
  void (*mixed_free)(void*) = nullptr;

  Profiler prof;

  size_t device_bytes = 0;
  std::vector<void*> allocations;

  int alloc(void** p, size_t bytes);
  ~Plan();
};

int apply_f64(Plan& P, const double* V, double* Out, cudaStream_t st);
int apply_combo_f64(Plan& P, const double* B, double* Out, cudaStream_t st);
int apply_mixed(Plan& P, const double* V, double* Out, cudaStream_t st);
// Reads and clears the device status word of the mixed path (synchronous).
int mixed_status(Plan& P, int* status);
int mixed_slices(const Plan& P);
// true if the plan's mixed apply folds Algorithm 1's weights into its last node pass
bool mixed_fused(const Plan& P);
// Prepares precision-specific plan state (no-op for FP64).
int precision_setup(Plan& P);
// Runs the apply for nrhs right-hand sides with the plan's precision.
int apply_dispatch(Plan& P, int nrhs, const double* V, double* Out, cudaStream_t st);

}  // namespace phikron

// The opaque handle of the C ABI.
struct phikron_plan_s {
  phikron::Plan impl;
};
