// C ABI of libphikron: plan construction (Algorithm 6's set-up) and the apply path
// (Algorithm 1 on 2^{-s}M, s modified-squaring steps of Eq. (29), phi_0 by Eq. (8)).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "checked.cuh"
#include "common.h"
#include "plan.h"

PK_CHK_BIND(api)

namespace phikron {

thread_local Profiler* tl_prof = nullptr;

namespace {
thread_local std::string g_err;
}

void set_error(const std::string& msg) { g_err = msg; }
void clear_error() { g_err.clear(); }

namespace {

struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  int rc = PHIKRON_OK;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      rc = PHIKRON_ECUDA;
      set_error("cudaGetDevice failed (no CUDA device?)");
      return;
    }
    if (dev >= 0 && dev != prev) {
      if (cudaSetDevice(dev) != cudaSuccess) {
        rc = PHIKRON_ECUDA;
        set_error("cudaSetDevice failed");
        return;
      }
      changed = true;
    }
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

double norm_inf(const double* a, int n) {
  double best = 0.0;
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += std::fabs(a[(size_t)i * n + j]);
    best = std::max(best, s);
  }
  return best;
}

double norm_one(const double* a, int n) {
  double best = 0.0;
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += std::fabs(a[(size_t)i * n + j]);
    best = std::max(best, s);
  }
  return best;
}

}  // namespace

Plan::~Plan() {
  for (cudaEvent_t e : {ev_in[0], ev_in[1], ev_comp[0], ev_comp[1], ev_out[0], ev_out[1], ev_start})
    if (e) cudaEventDestroy(e);
  if (cp_in) cudaStreamDestroy(cp_in);
  if (cp_out) cudaStreamDestroy(cp_out);
  for (void* p : allocations) device_free(p);
  if (mixed && mixed_free) mixed_free(mixed);
}

bool alloc_fault() {
  static std::mutex mu;
  static std::string seen;
  static long long count = 0;
  const char* v = std::getenv("PHIKRON_FAIL_ALLOC_AFTER");
  std::lock_guard<std::mutex> lock(mu);
  if (!v || !*v) {
    seen.clear();
    return false;
  }
  if (seen != v) {   // a new setting restarts the count
    seen = v;
    count = 0;
  }
  const long long k = std::atoll(v);
  return count++ >= k;
}

std::atomic<long long> g_live_buffers{0};

void device_free(void* p) {
  if (!p) return;
  chk::remove(p);
  cudaFree(p);
  g_live_buffers.fetch_sub(1);
}

int device_malloc(void** p, size_t bytes, const char* who) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (alloc_fault()) {
    set_error(std::string(who) + ": device allocation of " + std::to_string(bytes) +
              " bytes refused (PHIKRON_FAIL_ALLOC_AFTER)");
    return PHIKRON_ENOMEM;
  }
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_error(std::string(who) + ": cudaMalloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    return PHIKRON_ENOMEM;
  }
  g_live_buffers.fetch_add(1);
  chk::add(*p, bytes);
  return PHIKRON_OK;
}

int Plan::alloc(void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  PK_RET(device_malloc(p, bytes, "phikron_plan"));
  allocations.push_back(*p);
  device_bytes += bytes;
  return PHIKRON_OK;
}

int profiler_begin(Profiler& pr, int max_timed) {
  pr.launches = 0;
  for (int c = 0; c < KC_COUNT; ++c) pr.launches_by_class[c] = 0;
  pr.used = 0;
  while ((int)pr.cls.size() < max_timed) {
    cudaEvent_t a, b;
    PK_TRY_CUDA(cudaEventCreate(&a));
    PK_TRY_CUDA(cudaEventCreate(&b));
    pr.ev.push_back(a);
    pr.ev.push_back(b);
    pr.cls.push_back(0);
  }
  pr.timing = max_timed > 0;
  return PHIKRON_OK;
}

int profiler_end(Profiler& pr, phikron_profile* out) {
  for (int c = 0; c < KC_COUNT; ++c) out->launches[c] += pr.launches_by_class[c];
  for (size_t i = 0; i < pr.used; ++i) {
    PK_TRY_CUDA(cudaEventSynchronize(pr.ev[2 * i + 1]));
    float ms = 0.f;
    PK_TRY_CUDA(cudaEventElapsedTime(&ms, pr.ev[2 * i], pr.ev[2 * i + 1]));
    out->ms[pr.cls[i]] += ms;
  }
  out->timed_launches += (long long)pr.used;
  pr.timing = false;
  pr.used = 0;
  return PHIKRON_OK;
}

void selector_features(int dims, const int* n, const double* tau_norm_inf, int p, double tol, float* out) {
  for (int d = 0; d < 3; ++d) {
    if (d < dims) {
      out[d] = (float)std::log10(std::max(tau_norm_inf[d], 1e-30));
      out[3 + d] = (float)(std::log2((double)n[d]) / 8.0);
    } else {
      out[d] = -6.0f;
      out[3 + d] = 0.0f;
    }
  }
  out[6] = (float)(p / 4.0);
  out[7] = (float)(-std::log10(tol) / 10.0);
}

namespace {

bool is_symmetric(const double* a, int n) {
  double mx = 0.0;
  for (long long i = 0; i < (long long)n * n; ++i) mx = std::max(mx, std::fabs(a[i]));
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (std::fabs(a[(size_t)i * n + j] - a[(size_t)j * n + i]) > 1e-14 * mx) return false;
  return true;
}

// (s, m) from the learned selector with an a-posteriori check of the measured criterion over
// the Gershgorin interval of M = -tau*A; returns 1 (network), 2 (network, m raised until the
// check passes) or 3 (check failed: caller falls back to Algorithm 5).
int select_mlp(int dims, const double* const* A, const int* n, double tau, int l_max, double tol, int* s, int* m) {
  std::vector<float> params;
  if (!mlp::model(&params)) return -1;
  if (dims > 3) return 3;  // the network's features describe at most three factors
  double tn[3] = {0, 0, 0}, glo = 0.0, ghi = 0.0;
  bool sym = true;
  for (int d = 0; d < dims; ++d) {
    tn[d] = std::fabs(tau) * norm_inf(A[d], n[d]);
    sym = sym && is_symmetric(A[d], n[d]);
    double lo = INFINITY, hi = -INFINITY;
    for (int i = 0; i < n[d]; ++i) {
      double r = 0.0;
      for (int j = 0; j < n[d]; ++j)
        if (j != i) r += std::fabs(A[d][(size_t)i * n[d] + j]);
      lo = std::min(lo, A[d][(size_t)i * n[d] + i] - r);
      hi = std::max(hi, A[d][(size_t)i * n[d] + i] + r);
    }
    glo += lo;
    ghi += hi;
  }
  float feat[8];
  selector_features(dims, n, tn, l_max, tol, feat);
  float *dp = nullptr, *dx = nullptr;
  int* dsm = nullptr;
  int hs = 0, hm = 0;
  bool ok = cudaMalloc(&dp, sizeof(float) * params.size()) == cudaSuccess &&
            cudaMalloc(&dx, sizeof(float) * 8) == cudaSuccess && cudaMalloc(&dsm, sizeof(int) * 2) == cudaSuccess;
  ok = ok && cudaMemcpy(dp, params.data(), sizeof(float) * params.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaMemcpy(dx, feat, sizeof(float) * 8, cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && mlp::forward(dp, dx, 1, nullptr, dsm, dsm + 1, nullptr) == PHIKRON_OK;
  ok = ok && cudaMemcpy(&hs, dsm, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
  ok = ok && cudaMemcpy(&hm, dsm + 1, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
  cudaFree(dp);
  cudaFree(dx);
  cudaFree(dsm);
  if (!ok) {
    cudaGetLastError();
    return 3;
  }
  const double zlo = -std::fabs(tau) * ghi, zhi = -std::fabs(tau) * glo;
  if (!sym || zhi > 0.0 || !(zlo <= zhi)) return 3;  // outside the criterion's reach
  for (int extra = 0; extra <= 4 && hm + extra <= 32; ++extra) {
    if (selector::criterion(zlo, zhi, l_max, hs, hm + extra, 512) <= tol) {
      *s = hs;
      *m = hm + extra;
      return extra == 0 ? 1 : 2;
    }
  }
  return 3;
}

}  // namespace

// ----------------------------------------------------------------------------- plan

int build_plan(Plan& P, int dims, const double* const* A, const int* n, double tau, int l_max,
               double tol, const phikron_opts& o) {
  P.dims = dims;
  P.tau = tau;
  P.p = l_max;
  P.tol = tol;
  P.opts = o;
  P.N = 1;
  for (int d = 0; d < dims; ++d) {
    P.n[d] = n[d];
    P.N *= n[d];
  }
  for (int d = dims; d < PHIKRON_MAX_DIMS; ++d) P.n[d] = 1;
  for (int d = 0; d < PHIKRON_MAX_DIMS; ++d) P.pn[d] = P.n[d];
  P.PN = P.N;

  // alpha = tau * sum_d ||A^d||_inf  (Eq. (31))
  double alpha = 0.0;
  std::vector<double> n1(dims);
  for (int d = 0; d < dims; ++d) {
    alpha += std::fabs(tau) * norm_inf(A[d], n[d]);
    n1[d] = norm_one(A[d], n[d]);
  }
  if (o.alpha > 0.0) alpha = o.alpha;
  P.alpha = alpha;
  const double beta = (o.beta > 0.0) ? o.beta : 1.0;
  P.log10_bound = -INFINITY;

  // (s, m): Algorithm 5, unless forced or trivial.  Adaptive Clenshaw-Curtis (Algorithm 2)
  // takes s from Algorithm 5 with the CC bound and refines the node count at apply time.
  const bool adaptive = (o.quad == PHIKRON_QUAD_CC_ADAPTIVE);
  const int rule = adaptive ? PHIKRON_QUAD_CC : o.quad;
  int s = 0, m = 0, cost = 0;
  P.selector_used = PHIKRON_SELECT_PAPER;
  if (l_max >= 1) {
    int sel = 0;
    if (o.selector == PHIKRON_SELECT_MLP && alpha > 0.0 && o.quad == PHIKRON_QUAD_GAUSS) {
      sel = select_mlp(dims, A, n, tau, l_max, tol, &s, &m);
      if (sel < 0) {
        set_error("phikron_plan: PHIKRON_SELECT_MLP needs a selector model (phikron_selector_set_model or "
                  "phikron_selector_train)");
        return PHIKRON_EINVAL;
      }
      P.selector_used = (sel == 3) ? 3 : sel;
    }
    if (sel == 1 || sel == 2) {
      // (s, m) from the network, checked
    } else if (alpha > 0.0) {
      PK_RET(planner::setup_quadrature(tol, l_max, alpha, beta, rule, &s, &m, &cost));
    } else {
      s = 0;
      m = (l_max + 1) / 2 + 1;  // M = 0: the integrand is a polynomial of degree l_max-1
    }
    if (o.force_s >= 0) s = o.force_s;
    if (adaptive) {
      // levels l = 0..L with 6*2^l + 1 nodes (Algorithm 2 starts at n = 3: 2n + 1 = 7); the
      // cap is the first rule with at least twice the a-priori CC node count (force_m: at
      // least force_m nodes), never below one refinement and never above 385 nodes
      const int want = (o.force_m >= 1) ? o.force_m : 2 * m;
      int L = 1;
      while (L < 6 && 6 * (1 << L) + 1 < want) ++L;
      P.ad_levels = L;
      P.ad_nodes.clear();
      for (int l = 0; l <= L; ++l) P.ad_nodes.push_back(6 * (1 << l) + 1);
      m = P.ad_nodes.back();
    } else if (o.force_m >= 1) {
      m = o.force_m;
    }
    if (o.half_step && s < 1) s = 1;  // the half-step state is the one before the last squaring
    if (o.quad == PHIKRON_QUAD_CC && m < 2) m = 2;
    if ((m > 256 && !adaptive) || s > 60) {
      set_error("plan: node count or scaling out of range (m <= 256, s <= 60)");
      return PHIKRON_EINVAL;
    }
    if (alpha > 0.0) {
      double lb;
      if (planner::log_quaderr(std::max(1.0, (double)(m - 1)), l_max, std::ldexp(alpha, -s), beta,
                               rule, &lb) == PHIKRON_OK)
        P.log10_bound = lb / std::log(10.0);
      clear_error();
    }
  }
  P.s = s;
  P.m = m;
  P.cost = m + s * l_max;

  // quadrature rule and node weights c_{j,k} = w_k x_k^{j-1}/(j-1)!  (Algorithm 1)
  P.x.assign(m, 0.0);
  P.w.assign(m, 0.0);
  if (adaptive && l_max >= 1) {
    // nodes of the finest rule (n_f = 6*2^L intervals) in order of first appearance: level l
    // contributes the points j with j multiple of 2^{L-l} but not of 2^{L-l+1}
    const int L = P.ad_levels, nf = 6 << L;
    std::vector<double> xf(nf + 1), wf(nf + 1);
    PK_RET(planner::clenshaw_curtis(nf, xf.data(), wf.data()));
    std::vector<int> order;        // finest index of each stored node
    for (int l = 0; l <= L; ++l) {
      const int step = 1 << (L - l);
      for (int j = 0; j <= nf; j += step)
        if (l == 0 || (j / step) % 2 == 1) order.push_back(j);
    }
    for (int k = 0; k < m; ++k) {
      P.x[k] = xf[order[k]];
      P.w[k] = wf[order[k]];
    }
    // weights of every level's rule over its stored nodes: c_{j,k} = w_k^{(l)} x_k^{j-1}/(j-1)!
    P.coef.clear();
    P.ad_coef_off.clear();
    for (int l = 0; l <= L; ++l) {
      const int nl = 6 << l, cnt = P.ad_nodes[l], step = 1 << (L - l);
      std::vector<double> xl(nl + 1), wl(nl + 1);
      PK_RET(planner::clenshaw_curtis(nl, xl.data(), wl.data()));
      P.ad_coef_off.push_back(P.coef.size());
      const size_t base = P.coef.size();
      P.coef.resize(base + (size_t)l_max * cnt);
      for (int j = 1; j <= l_max; ++j) {
        double fact = 1.0;
        for (int q = 2; q <= j - 1; ++q) fact *= q;
        for (int k = 0; k < cnt; ++k) {
          const int jl = order[k] / step;  // index of stored node k in the level-l rule
          P.coef[base + (size_t)(j - 1) * cnt + k] = wl[jl] * std::pow(xl[jl], j - 1) / fact;
        }
      }
    }
  } else {
    if (m > 0) {
      if (o.quad == PHIKRON_QUAD_GAUSS)
        PK_RET(planner::gauss_legendre(m, P.x.data(), P.w.data()));
      else
        PK_RET(planner::clenshaw_curtis(m - 1, P.x.data(), P.w.data()));
    }
    P.coef.assign((size_t)std::max(1, l_max) * std::max(1, m), 0.0);
    for (int j = 1; j <= l_max; ++j) {
      double fact = 1.0;
      for (int q = 2; q <= j - 1; ++q) fact *= q;
      for (int k = 0; k < m; ++k) P.coef[(size_t)(j - 1) * m + k] = P.w[k] * std::pow(P.x[k], j - 1) / fact;
    }
  }

  // unique factors (bitwise-equal matrices share their exponentials)
  P.nuniq = 0;
  for (int d = 0; d < dims; ++d) {
    int found = -1;
    for (int u = 0; u < P.nuniq; ++u) {
      const int dd = P.uniq_rep[u];
      if (n[dd] == n[d] && std::memcmp(A[dd], A[d], sizeof(double) * (size_t)n[d] * n[d]) == 0) {
        found = u;
        break;
      }
    }
    if (found < 0) {
      found = P.nuniq++;
      P.uniq_rep[found] = d;
    }
    P.uniq_of[d] = found;
  }

  // device: 1D exponentials per unique factor, layout [nodes 0..m-1 | G_s | G_0..G_{s-1}]
  P.nexp = m + 1 + s;
  cudaStream_t st = nullptr;
  for (int u = 0; u < P.nuniq; ++u) {
    const int d = P.uniq_rep[u];
    const int nd = n[d];
    const size_t nn = (size_t)nd * nd;
    const int cnt = m + 1 + (s > 0 ? 1 : 0);  // nodes, exp(M), G_0
    double* dExp = nullptr;
    PK_RET(P.alloc((void**)&dExp, sizeof(double) * nn * P.nexp));
    P.dExp[u] = dExp;
    double* dIn = nullptr;
    void* ws = nullptr;
    double* dOut = nullptr;
    PK_RET(P.alloc((void**)&dIn, sizeof(double) * nn * cnt));
    PK_RET(P.alloc((void**)&dOut, sizeof(double) * nn * cnt));
    PK_RET(P.alloc(&ws, expm_workspace_bytes(cnt, nd)));
    for (int c = 0; c < cnt; ++c)
      PK_TRY_CUDA(cudaMemcpy(dIn + c * nn, A[d], sizeof(double) * nn, cudaMemcpyHostToDevice));
    std::vector<double> scale(cnt), norms(cnt, n1[d]);
    const double sc = -tau * std::ldexp(1.0, -s);
    for (int k = 0; k < m; ++k) scale[k] = sc * (1.0 - P.x[k]);
    scale[m] = -tau;  // exp(M^d) for phi_0
    if (s > 0) scale[m + 1] = sc;  // G_0 = exp(2^{-s} M^d)
    PK_RET(expm_batched(cnt, nd, dIn, scale.data(), norms.data(), dOut, ws, st));
    PK_TRY_CUDA(cudaMemcpyAsync(dExp, dOut, sizeof(double) * nn * (m + 1), cudaMemcpyDeviceToDevice, st));
    if (s > 0) {
      PK_TRY_CUDA(cudaMemcpyAsync(dExp + (size_t)(m + 1) * nn, dOut + (size_t)(m + 1) * nn,
                                  sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
      // G_{t+1} = G_t^2  (Algorithm 6, step 2 of the squaring loop)
      for (int t = 0; t + 1 < s; ++t) {
        GemmF64 g{};
        const double* Gt = dExp + (size_t)(m + 1 + t) * nn;
        double* Gn = dExp + (size_t)(m + 2 + t) * nn;
        g.A = Gt; g.sAm = nd; g.sAk = 1;
        g.B = Gt; g.sBk = nd; g.sBn = 1;
        g.C = Gn; g.sCm = nd; g.sCn = 1;
        g.M = g.N = g.K = nd; g.nb = 1; g.nb0 = 1; g.alpha = 1.0; g.beta = 0.0;
        PK_RET(gemm_f64(g, st));
      }
    }
    PK_TRY_CUDA(cudaStreamSynchronize(st));
    // staging for the expm is no longer needed
    for (void* q : {(void*)dIn, (void*)dOut, ws}) {
      device_free(q);
      P.allocations.erase(std::find(P.allocations.begin(), P.allocations.end(), q));
    }
    P.device_bytes -= sizeof(double) * nn * cnt * 2 + expm_workspace_bytes(cnt, nd);
  }

  // node weights on the device
  PK_RET(P.alloc((void**)&P.dCoef, sizeof(double) * P.coef.size()));
  PK_TRY_CUDA(cudaMemcpy(P.dCoef, P.coef.data(), sizeof(double) * P.coef.size(), cudaMemcpyHostToDevice));

  // apply work buffers
  const long long N = P.N;
  int nv = std::max(m + 2, std::max(l_max, 1));
  if (P.ad_levels >= 0) {
    // node vectors kept across refinements; the mode chain of one level needs room for its
    // new nodes only
    nv = std::max(P.ad_nodes[P.ad_levels] - P.ad_nodes[P.ad_levels - 1] + 2, std::max(l_max, 1));
    PK_RET(P.alloc((void**)&P.dT, sizeof(double) * (size_t)m * N));
    PK_RET(P.alloc((void**)&P.dErr, sizeof(unsigned long long) * 2 * (size_t)l_max));
  }
  PK_RET(P.alloc((void**)&P.dW1, sizeof(double) * (size_t)nv * N));
  PK_RET(P.alloc((void**)&P.dW2, sizeof(double) * (size_t)nv * N));
  PK_RET(P.alloc((void**)&P.dY, sizeof(double) * (size_t)std::max(l_max, 1) * N));
  PK_RET(P.alloc((void**)&P.dYn, sizeof(double) * (size_t)std::max(l_max, 1) * N));
  PK_RET(P.alloc((void**)&P.dV, sizeof(double) * (size_t)N));
  PK_RET(P.alloc((void**)&P.dOut, sizeof(double) * (size_t)(l_max + 1) * (o.half_step ? 2 : 1) * N));
  if (s == 0 && l_max >= 1 && m > 0 && o.precision == PHIKRON_PREC_FP64 && P.ad_levels < 0) {
    // tables and buffer of phikron_apply_combo: [m x l_max] x_i^{j-1}/(j-1)!, then [m] w_i
    std::vector<double> cb((size_t)m * l_max + m);
    for (int i = 0; i < m; ++i) {
      double t = 1.0;
      for (int j = 1; j <= l_max; ++j) {
        cb[(size_t)i * l_max + (j - 1)] = t;
        t = t * P.x[i] / j;
      }
      cb[(size_t)m * l_max + i] = P.w[i];
    }
    PK_RET(P.alloc((void**)&P.dCombo, sizeof(double) * cb.size()));
    PK_TRY_CUDA(cudaMemcpy(P.dCombo, cb.data(), sizeof(double) * cb.size(), cudaMemcpyHostToDevice));
    PK_RET(P.alloc((void**)&P.dY2, sizeof(double) * (size_t)m * N));
  }
  PK_RET(precision_setup(P));
  return PHIKRON_OK;
}

// (x)_d E_d applied to `nvec` vectors, each with its own matrices (E_stride matrices apart
// in the per-factor exponential arrays, starting at index e0) or shared ones (E_stride 0).
// src -> ... -> result; returns the buffer holding the result.
int kron_chain_f64(const Plan& P, const double* src, long long src_sb, int nvec, int e0, int e_stride,
                   double* bufA, double* bufB, double* final_dst, cudaStream_t st) {
  const long long N = P.N;
  const double* cur = src;
  long long cur_sb = src_sb;
  for (int d = 0; d < P.dims; ++d) {
    long long B0 = 1, R = 1;
    for (int q = 0; q < d; ++q) B0 *= P.n[q];
    for (int q = d + 1; q < P.dims; ++q) R *= P.n[q];
    const int nd = P.n[d];
    const size_t nn = (size_t)nd * nd;
    const double* E = P.dExp[P.uniq_of[d]] + (size_t)e0 * nn;
    double* dst = (d == P.dims - 1) ? final_dst : ((d % 2 == 0) ? bufA : bufB);
    PK_RET(mode_product_f64(cur, cur_sb, dst, N, E, (long long)e_stride * nn, nvec, B0, nd, R, st));
    cur = dst;
    cur_sb = N;
  }
  return PHIKRON_OK;
}

// Algorithm 2's error: max_j ||y_j - y~_j||_inf / ||y_j||_inf; slots[2j] and slots[2j+1] receive
// the bit patterns of max|y_j - y~_j| and max|y_j| (non-negative doubles order like integers)
__global__ void cc_err_kernel(const double* __restrict__ Y, const double* __restrict__ Yo, int p, long long N,
                              unsigned long long* __restrict__ slots) {
  for (int j = 0; j < p; ++j) {
    double dmax = 0.0, ymax = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
      const double y = chk::ld_ck(Y + (size_t)j * N + i, chk::SITE_PLAN);
      dmax = fmax(dmax, fabs(y - chk::ld_ck(Yo + (size_t)j * N + i, chk::SITE_PLAN)));
      ymax = fmax(ymax, fabs(y));
    }
    for (int o = 16; o > 0; o >>= 1) {
      dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      ymax = fmax(ymax, __shfl_xor_sync(0xffffffffu, ymax, o));
    }
    if ((threadIdx.x & 31) == 0) {
      if (PK_CK(slots + 2 * j, 2 * sizeof(unsigned long long), chk::SITE_PLAN)) {
        atomicMax(slots + 2 * j, (unsigned long long)__double_as_longlong(dmax));
        atomicMax(slots + 2 * j + 1, (unsigned long long)__double_as_longlong(ymax));
      }
    }
  }
}

// Algorithm 3 with Algorithm 2: nested Clenshaw-Curtis rules on 2^{-s}M, refined until the
// max-norm change of every y_j is <= tol relative, then the s squaring steps.
int apply_f64_adaptive(Plan& P, const double* V, double* Out, cudaStream_t st) {
  const long long N = P.N;
  const int p = P.p, m = P.m, s = P.s, L = P.ad_levels;
  if (!P.opts.skip_phi0) PK_RET(kron_chain_f64(P, V, 0, 1, m, 0, P.dW1, P.dW2, Out, st));
  double* bufs[2] = {P.dY, P.dYn};
  int cur = 0, done = 0;
  double err = INFINITY;
  int used = 0;
  for (int l = 0; l <= L; ++l) {
    const int nl = P.ad_nodes[l];
    // v_i = e^{(1 - x_i) 2^{-s} M} v for the nodes this rule adds (stored after the earlier ones)
    PK_RET(kron_chain_f64(P, V, 0, nl - done, done, 1, P.dW1, P.dW2, P.dT + (size_t)done * N, st));
    done = nl;
    used = nl;
    PK_RET(weighted_sum_f64(P.dT, N, P.dCoef + P.ad_coef_off[l], p, nl, N, bufs[cur], N, st));
    if (l >= 1) {
      PK_TRY_CUDA(cudaMemsetAsync(P.dErr, 0, sizeof(unsigned long long) * 2 * p, st));
      cc_err_kernel<<<(int)std::min<long long>((N + 255) / 256, 152 * 4), 256, 0, st>>>(bufs[cur], bufs[cur ^ 1], p,
                                                                                      N, P.dErr);
      PK_CHECK_LAUNCH();
      std::vector<unsigned long long> h(2 * p);
      PK_TRY_CUDA(cudaMemcpyAsync(h.data(), P.dErr, sizeof(unsigned long long) * 2 * p, cudaMemcpyDeviceToHost, st));
      PK_TRY_CUDA(cudaStreamSynchronize(st));
      err = 0.0;
      for (int j = 0; j < p; ++j) {
        double dm, ym;
        std::memcpy(&dm, &h[2 * j], sizeof(double));
        std::memcpy(&ym, &h[2 * j + 1], sizeof(double));
        // a zero y_j with a zero change counts as converged
        err = std::max(err, (ym > 0.0) ? dm / ym : (dm > 0.0 ? INFINITY : 0.0));
      }
      if (err <= P.tol) break;
    }
    cur ^= 1;
  }
  if (!(err <= P.tol)) cur ^= 1;  // the loop left cur one past the last level's buffer
  P.last_nodes = used;
  P.last_err = err;
  double* Y = bufs[cur];
  double* Yn = bufs[cur ^ 1];
  if (s == 0) {
    PK_TRY_CUDA(cudaMemcpyAsync(Out + N, Y, sizeof(double) * (size_t)p * N, cudaMemcpyDeviceToDevice, st));
  } else {
    for (int t = 0; t < s; ++t) {
      double* Z = (P.dims % 2 == 1) ? P.dW1 : P.dW2;
      PK_RET(kron_chain_f64(P, Y, N, p, m + 1 + t, 0, P.dW1, P.dW2, Z, st));
      double* dst = (t == s - 1) ? Out + N : Yn;
      PK_RET(squaring_combine_f64(Z, Y, dst, p, N, N, st));
      Yn = Y;
      Y = dst;
    }
  }
  if (!(err <= P.tol)) {
    set_error("adaptive Clenshaw-Curtis: not converged at the node cap (Out holds the cap's result)");
    return PHIKRON_ENOTCONVERGED;
  }
  return PHIKRON_OK;
}

// The Remark after Algorithm 2: sum_j phi_j(M) b_j ~ sum_i w_i e^{(1-x_i)M} z_i with
// z_i = sum_j x_i^{j-1}/(j-1)! b_j (s = 0).  P.dCombo holds the m x p table x_i^{j-1}/(j-1)!
// followed by the m weights w_i.
int apply_combo_f64(Plan& P, const double* B, double* Out, cudaStream_t st) {
  const long long N = P.N;
  const int p = P.p, m = P.m;
  double* Z = P.dY2;                                     // m vectors z_i
  double* T = (P.dims % 2 == 1) ? P.dW1 : P.dW2;         // m vectors e^{(1-x_i)M} z_i
  for (int c = 0; c < m; c += 20)  // the weighted-sum kernel forms at most 20 outputs per launch
    PK_RET(weighted_sum_f64(B, N, P.dCombo + (size_t)c * p, std::min(20, m - c), p, N, Z + (size_t)c * N, N, st));
  PK_RET(kron_chain_f64(P, Z, N, m, 0, 1, P.dW1, P.dW2, T, st));
  return weighted_sum_f64(T, N, P.dCombo + (size_t)m * p, 1, m, N, Out, N, st);
}

int apply_f64(Plan& P, const double* V, double* Out, cudaStream_t st) {
  const long long N = P.N;
  const int p = P.p, m = P.m, s = P.s;
  if (P.ad_levels >= 0 && p >= 1) return apply_f64_adaptive(P, V, Out, st);
  if (p == 0) {
    // phi_0 only: (x)_d exp(M^d) v
    return kron_chain_f64(P, V, 0, 1, m, 0, P.dW1, P.dW2, Out, st);
  }
  // node phase: m node actions + phi_0 in one batched chain (v shared: stride 0)
  const bool phi0 = !P.opts.skip_phi0;
  PK_RET(kron_chain_f64(P, V, 0, m + (phi0 ? 1 : 0), 0, 1, P.dW1, P.dW2,
                        (P.dims % 2 == 1) ? P.dW1 : P.dW2, st));
  const double* T = (P.dims % 2 == 1) ? P.dW1 : P.dW2;
  // the chain's last destination is the buffer given; use a dedicated one to avoid aliasing
  if (phi0)
    PK_TRY_CUDA(cudaMemcpyAsync(Out, T + (size_t)m * N, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
  double* Y = (s == 0) ? Out + N : P.dY;
  PK_RET(weighted_sum_f64(T, N, P.dCoef, p, m, N, Y, N, st));
  double* Yn = P.dYn;
  for (int t = 0; t < s; ++t) {
    // Z_i = (x)_d G_{t,d} y_i for i = 1..p (shared matrices)
    double* Z = (P.dims % 2 == 1) ? P.dW1 : P.dW2;
    PK_RET(kron_chain_f64(P, Y, N, p, m + 1 + t, 0, P.dW1, P.dW2, Z, st));
    double* dst = (t == s - 1) ? Out + N : Yn;
    PK_RET(squaring_combine_f64(Z, Y, dst, p, N, N, st));
    Yn = Y;
    Y = dst;
  }
  return PHIKRON_OK;
}

}  // namespace phikron

// =============================================================================== C ABI
using namespace phikron;


extern "C" {

void phikron_opts_default(phikron_opts* o) {
  if (!o) return;
  o->quad = PHIKRON_QUAD_GAUSS;
  o->precision = PHIKRON_PREC_FP64;
  o->selector = PHIKRON_SELECT_PAPER;
  o->force_s = -1;
  o->force_m = -1;
  o->alpha = 0.0;
  o->beta = 0.0;
  o->device = -1;
  o->max_rhs = 1;
  o->slices = 0;
  o->half_step = 0;
  o->skip_phi0 = 0;
  o->wait_us = 0;
}

const char* phikron_last_error(void) { return g_err.c_str(); }

long long phikron_live_device_buffers(void) { return phikron::g_live_buffers.load(); }

int phikron_plan(phikron_plan_t* out, int dims, const double* const* A, const int* n, double tau,
                 int l_max, double tol, const phikron_opts* opts) {
  clear_error();
  if (!out) { set_error("phikron_plan: out is NULL"); return PHIKRON_EINVAL; }
  *out = nullptr;
  if (dims < 1 || dims > PHIKRON_MAX_DIMS) { set_error("phikron_plan: dims must be in 1..PHIKRON_MAX_DIMS"); return PHIKRON_EINVAL; }
  if (!A || !n) { set_error("phikron_plan: A or n is NULL"); return PHIKRON_EINVAL; }
  if (!std::isfinite(tau)) { set_error("phikron_plan: tau must be finite"); return PHIKRON_EINVAL; }
  if (l_max < 0 || l_max > 20) { set_error("phikron_plan: l_max must be in 0..20"); return PHIKRON_EINVAL; }
  if (!(tol >= 1e-16 && tol < 1.0)) { set_error("phikron_plan: tol must be in [1e-16, 1)"); return PHIKRON_EINVAL; }
  long long N = 1;
  for (int d = 0; d < dims; ++d) {
    if (!A[d]) { set_error("phikron_plan: factor pointer is NULL"); return PHIKRON_EINVAL; }
    if (n[d] < 1 || n[d] > 4096) { set_error("phikron_plan: n[d] must be in 1..4096"); return PHIKRON_EINVAL; }
    for (long long i = 0; i < (long long)n[d] * n[d]; ++i)
      if (!std::isfinite(A[d][i])) { set_error("phikron_plan: factor has NaN/Inf"); return PHIKRON_EINVAL; }
    N *= n[d];
  }
  if (N > (1LL << 31)) { set_error("phikron_plan: N = prod n[d] must be <= 2^31"); return PHIKRON_EINVAL; }
  phikron_opts o;
  phikron_opts_default(&o);
  if (opts) o = *opts;
  if (o.quad != PHIKRON_QUAD_GAUSS && o.quad != PHIKRON_QUAD_CC && o.quad != PHIKRON_QUAD_CC_ADAPTIVE) {
    set_error("phikron_plan: bad quad");
    return PHIKRON_EINVAL;
  }
  if (o.quad == PHIKRON_QUAD_CC_ADAPTIVE && o.precision != PHIKRON_PREC_FP64) {
    set_error("phikron_plan: adaptive Clenshaw-Curtis runs on the float64 path");
    return PHIKRON_ENOTSUP;
  }
  if (o.precision != PHIKRON_PREC_FP64 && o.precision != PHIKRON_PREC_OZAKI_BF16) { set_error("phikron_plan: bad precision"); return PHIKRON_EINVAL; }
  if (o.max_rhs < 1) o.max_rhs = 1;
  if (o.half_step && o.precision != PHIKRON_PREC_OZAKI_BF16) {
    set_error("phikron_plan: half_step outputs are built for the mixed path only");
    return PHIKRON_ENOTSUP;
  }
  if (o.half_step && l_max == 0) {
    set_error("phikron_plan: half_step needs l_max >= 1");
    return PHIKRON_EINVAL;
  }
  if (o.skip_phi0 && l_max == 0) {
    set_error("phikron_plan: skip_phi0 needs l_max >= 1");
    return PHIKRON_EINVAL;
  }
  if (o.selector != PHIKRON_SELECT_PAPER && o.selector != PHIKRON_SELECT_MLP) {
    set_error("phikron_plan: bad selector");
    return PHIKRON_EINVAL;
  }
  if (o.wait_us < 0) {
    set_error("phikron_plan: wait_us must be >= 0");
    return PHIKRON_EINVAL;
  }
  DeviceGuard dg(o.device);
  if (dg.rc != PHIKRON_OK) return dg.rc;
  if (cudaGetDevice(&o.device) != cudaSuccess) { set_error("cudaGetDevice failed"); return PHIKRON_ECUDA; }
  phikron_plan_s* h = alloc_fault() ? nullptr : new (std::nothrow) phikron_plan_s();
  if (!h) { set_error("phikron_plan: host allocation failed"); return PHIKRON_ENOMEM; }
  int rc;
  try {
    rc = build_plan(h->impl, dims, A, n, tau, l_max, tol, o);
  } catch (const std::bad_alloc&) {
    set_error("phikron_plan: host allocation failed");
    rc = PHIKRON_ENOMEM;
  }
  if (rc != PHIKRON_OK) {
    delete h;
    return rc;
  }
  *out = h;
  return PHIKRON_OK;
}

// bytes of the Out buffer of nrhs applies: (l_max+1) vectors per rhs, twice with half_step
static size_t apply_out_bytes(const Plan& P, int nrhs) {
  return sizeof(double) * (size_t)P.N * (size_t)(P.p + 1) * (P.opts.half_step ? 2 : 1) * (size_t)nrhs;
}

int phikron_apply(phikron_plan_t plan, const double* V, double* Out, void* stream) {
  clear_error();
  if (!plan || !V || !Out) { set_error("phikron_apply: NULL argument"); return PHIKRON_EINVAL; }
  Plan& P = plan->impl;
  DeviceGuard dg(P.opts.device);
  if (dg.rc != PHIKRON_OK) return dg.rc;
  ProfScope ps(&P.prof);
  const chk::Range r[2] = {{V, sizeof(double) * (size_t)P.N}, {Out, apply_out_bytes(P, 1)}};
  chk::CallScope cs(static_cast<cudaStream_t>(stream), r, 2);
  PK_RET(cs.rc);
  return apply_dispatch(P, 1, V, Out, static_cast<cudaStream_t>(stream));
}

int phikron_apply_many(phikron_plan_t plan, int nrhs, const double* V, double* Out, void* stream) {
  clear_error();
  if (!plan || !V || !Out) { set_error("phikron_apply_many: NULL argument"); return PHIKRON_EINVAL; }
  Plan& P = plan->impl;
  if (nrhs < 1 || nrhs > P.opts.max_rhs) { set_error("phikron_apply_many: nrhs out of range"); return PHIKRON_EINVAL; }
  DeviceGuard dg(P.opts.device);
  if (dg.rc != PHIKRON_OK) return dg.rc;
  ProfScope ps(&P.prof);
  const chk::Range r[2] = {{V, sizeof(double) * (size_t)P.N * nrhs}, {Out, apply_out_bytes(P, nrhs)}};
  chk::CallScope cs(static_cast<cudaStream_t>(stream), r, 2);
  PK_RET(cs.rc);
  return apply_dispatch(P, nrhs, V, Out, static_cast<cudaStream_t>(stream));
}

int phikron_apply_combo(phikron_plan_t plan, const double* B, double* Out, void* stream) {
  clear_error();
  if (!plan || !B || !Out) { set_error("phikron_apply_combo: NULL argument"); return PHIKRON_EINVAL; }
  Plan& P = plan->impl;
  if (P.opts.precision != PHIKRON_PREC_FP64 || P.ad_levels >= 0) {
    set_error("phikron_apply_combo: runs on float64 plans with a fixed rule");
    return PHIKRON_ENOTSUP;
  }
  if (P.s != 0 || P.p < 1 || !P.dCombo) {
    set_error("phikron_apply_combo: needs a plan with s = 0 and l_max >= 1 (the combination does not "
              "commute with the modified squaring)");
    return PHIKRON_EINVAL;
  }
  DeviceGuard dg(P.opts.device);
  if (dg.rc != PHIKRON_OK) return dg.rc;
  ProfScope ps(&P.prof);
  const chk::Range r[2] = {{B, sizeof(double) * (size_t)P.N * P.p}, {Out, sizeof(double) * (size_t)P.N}};
  chk::CallScope cs(static_cast<cudaStream_t>(stream), r, 2);
  PK_RET(cs.rc);
  return apply_combo_f64(P, B, Out, static_cast<cudaStream_t>(stream));
}

// Pipelined host-buffer applies: vector j is applied on `stream` from staging buffer j % 2
// while vector j + 1 is copied in on one copy stream and the results of vector j - 1 are
// copied out on another, so that both link directions and the GPU are busy at once.
// Events order each reuse of a staging buffer after the work that last touched it.
static int host_many_enqueue(Plan& P, const double* V_host, double* Out_host, int count, cudaStream_t st) {
  chk::CallScope cs(st, nullptr, 0);   // device work on the plan's own staging buffers only
  PK_RET(cs.rc);
  const size_t in_elems = (size_t)P.N;
  const size_t out_elems = (size_t)P.N * (P.p + 1) * (P.opts.half_step ? 2 : 1);
  if (!P.dV2) {
    PK_RET(P.alloc((void**)&P.dV2, sizeof(double) * in_elems));
    PK_RET(P.alloc((void**)&P.dOut2, sizeof(double) * out_elems));
    PK_TRY_CUDA(cudaStreamCreateWithFlags(&P.cp_in, cudaStreamNonBlocking));
    PK_TRY_CUDA(cudaStreamCreateWithFlags(&P.cp_out, cudaStreamNonBlocking));
    for (cudaEvent_t* e : {&P.ev_in[0], &P.ev_in[1], &P.ev_comp[0], &P.ev_comp[1], &P.ev_out[0], &P.ev_out[1], &P.ev_start})
      PK_TRY_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  }
  double* Vd[2] = {P.dV, P.dV2};
  double* Od[2] = {P.dOut, P.dOut2};
  // the copy streams start after whatever the caller queued on `stream` before this call
  PK_TRY_CUDA(cudaEventRecord(P.ev_start, st));
  PK_TRY_CUDA(cudaStreamWaitEvent(P.cp_in, P.ev_start, 0));
  PK_TRY_CUDA(cudaStreamWaitEvent(P.cp_out, P.ev_start, 0));
  for (int j = 0; j < count; ++j) {
    const int b = j & 1;
    // staging input b was last read by the apply of vector j - 2
    if (j >= 2) PK_TRY_CUDA(cudaStreamWaitEvent(P.cp_in, P.ev_comp[b], 0));
    PK_TRY_CUDA(cudaMemcpyAsync(Vd[b], V_host + (size_t)j * in_elems, sizeof(double) * in_elems,
                                cudaMemcpyHostToDevice, P.cp_in));
    PK_TRY_CUDA(cudaEventRecord(P.ev_in[b], P.cp_in));
    // the apply needs its input, and staging output b must have been copied out (vector j - 2)
    PK_TRY_CUDA(cudaStreamWaitEvent(st, P.ev_in[b], 0));
    if (j >= 2) PK_TRY_CUDA(cudaStreamWaitEvent(st, P.ev_out[b], 0));
    {
      ProfScope ps(&P.prof);
      PK_RET(apply_dispatch(P, 1, Vd[b], Od[b], st));
    }
    PK_TRY_CUDA(cudaEventRecord(P.ev_comp[b], st));
    PK_TRY_CUDA(cudaStreamWaitEvent(P.cp_out, P.ev_comp[b], 0));
    PK_TRY_CUDA(cudaMemcpyAsync(Out_host + (size_t)j * out_elems, Od[b], sizeof(double) * out_elems,
                                cudaMemcpyDeviceToHost, P.cp_out));
    PK_TRY_CUDA(cudaEventRecord(P.ev_out[b], P.cp_out));
  }
  // `stream` is ordered after the last copy-out
  PK_TRY_CUDA(cudaStreamWaitEvent(st, P.ev_out[(count - 1) & 1], 0));
  return PHIKRON_OK;
}

int phikron_apply_host_many(phikron_plan_t plan, const double* V_host, double* Out_host, int count, void* stream) {
  clear_error();
  if (!plan || !V_host || !Out_host || count < 1) {
    set_error("phikron_apply_host_many: NULL argument or count < 1");
    return PHIKRON_EINVAL;
  }
  Plan& P = plan->impl;
  DeviceGuard dg(P.opts.device);
  if (dg.rc != PHIKRON_OK) return dg.rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int rc = host_many_enqueue(P, V_host, Out_host, count, st);
  // whatever was enqueued (on success or after an error) finishes before the host buffers
  // are handed back
  const cudaError_t e0 = cudaStreamSynchronize(st);
  const cudaError_t e1 = P.cp_in ? cudaStreamSynchronize(P.cp_in) : cudaSuccess;
  const cudaError_t e2 = P.cp_out ? cudaStreamSynchronize(P.cp_out) : cudaSuccess;
  if (rc != PHIKRON_OK) return rc;
  for (cudaError_t e : {e0, e1, e2}) {
    if (e != cudaSuccess) {
      set_error(std::string("phikron_apply_host_many: ") + cudaGetErrorString(e));
      return PHIKRON_ECUDA;
    }
  }
  return PHIKRON_OK;
}

int phikron_apply_host(phikron_plan_t plan, const double* V_host, double* Out_host, void* stream) {
  clear_error();
  if (!plan || !V_host || !Out_host) { set_error("phikron_apply_host: NULL argument"); return PHIKRON_EINVAL; }
  Plan& P = plan->impl;
  DeviceGuard dg(P.opts.device);
  if (dg.rc != PHIKRON_OK) return dg.rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  PK_TRY_CUDA(cudaMemcpyAsync(P.dV, V_host, sizeof(double) * P.N, cudaMemcpyHostToDevice, st));
  int rc;
  {
    ProfScope ps(&P.prof);
    rc = apply_dispatch(P, 1, P.dV, P.dOut, st);
  }
  if (rc != PHIKRON_OK) {
    cudaStreamSynchronize(st);  // the copy from V_host is done before V_host goes back
    return rc;
  }
  PK_TRY_CUDA(cudaMemcpyAsync(Out_host, P.dOut, sizeof(double) * P.N * (P.p + 1) * (P.opts.half_step ? 2 : 1),
                              cudaMemcpyDeviceToHost, st));
  PK_TRY_CUDA(cudaStreamSynchronize(st));
  return PHIKRON_OK;
}

int phikron_plan_info(phikron_plan_t plan, phikron_info* info) {
  clear_error();
  if (!plan || !info) { set_error("phikron_plan_info: NULL argument"); return PHIKRON_EINVAL; }
  const Plan& P = plan->impl;
  std::memset(info, 0, sizeof(*info));
  info->dims = P.dims;
  for (int d = 0; d < PHIKRON_MAX_DIMS; ++d) info->n[d] = P.n[d];
  info->N = P.N;
  info->l_max = P.p;
  info->s = P.s;
  info->m = P.m;
  info->cost = P.cost;
  const int nodes = (P.ad_levels >= 0 && P.last_nodes > 0) ? P.last_nodes : P.m;  // adaptive: last apply
  info->actions = (P.p == 0) ? 1 : nodes + P.s * P.p + (P.opts.skip_phi0 ? 0 : 1);
  info->alpha = P.alpha;
  info->log10_bound = P.log10_bound;
  info->precision = P.opts.precision;
  info->quad = P.opts.quad;
  info->selector_used = P.selector_used;
  info->unique_factors = P.nuniq;
  info->device_bytes = P.device_bytes;
  info->adaptive_nodes = P.last_nodes;
  info->adaptive_err = P.last_err;
  info->slices = P.mixed ? mixed_slices(P) : 0;
  info->fused_weights = mixed_fused(P) ? 1 : 0;
  return PHIKRON_OK;
}

int phikron_plan_nodes(phikron_plan_t plan, double* x, double* w) {
  clear_error();
  if (!plan || !x || !w) { set_error("phikron_plan_nodes: NULL argument"); return PHIKRON_EINVAL; }
  const Plan& P = plan->impl;
  for (int k = 0; k < P.m; ++k) {
    x[k] = P.x[k];
    w[k] = P.w[k];
  }
  return PHIKRON_OK;
}

void phikron_destroy(phikron_plan_t plan) { delete plan; }

int phikron_check_status(phikron_plan_t plan) {
  clear_error();
  if (!plan) { set_error("phikron_check_status: NULL plan"); return PHIKRON_EINVAL; }
  DeviceGuard dg(plan->impl.opts.device);
  if (dg.rc != PHIKRON_OK) return dg.rc;
  PK_TRY_CUDA(cudaDeviceSynchronize());
  PK_RET(chk::status());   // bounds-checked build: a recorded out-of-range access
  int st = 0;
  PK_RET(mixed_status(plan->impl, &st));
  if (st != 0) {
    set_error("a bounded device wait expired during an earlier apply");
    return st;
  }
  return PHIKRON_OK;
}

int phikron_profile_begin(phikron_plan_t plan, int max_timed) {
  clear_error();
  if (!plan || max_timed < 0) { set_error("phikron_profile_begin: bad arguments"); return PHIKRON_EINVAL; }
  DeviceGuard dg(plan->impl.opts.device);
  if (dg.rc != PHIKRON_OK) return dg.rc;
  return profiler_begin(plan->impl.prof, max_timed);
}

int phikron_profile_end(phikron_plan_t plan, phikron_profile* out) {
  clear_error();
  if (!plan || !out) { set_error("phikron_profile_end: NULL argument"); return PHIKRON_EINVAL; }
  DeviceGuard dg(plan->impl.opts.device);
  if (dg.rc != PHIKRON_OK) return dg.rc;
  std::memset(out, 0, sizeof(*out));
  return profiler_end(plan->impl.prof, out);
}

int phikron_log_quaderr(double n, int p, double alpha, double beta, int rule, double* log_err) {
  clear_error();
  if (!log_err) { set_error("phikron_log_quaderr: NULL output"); return PHIKRON_EINVAL; }
  return planner::log_quaderr(n, p, alpha, beta, rule, log_err);
}

int phikron_quadnodes(double eps, int p, double alpha, double beta, int rule, int* n) {
  clear_error();
  if (!n) { set_error("phikron_quadnodes: NULL output"); return PHIKRON_EINVAL; }
  return planner::quadnodes(eps, p, alpha, beta, rule, n);
}

int phikron_setup_quadrature(double eps, int p, double alpha, double beta, int rule, int* s, int* m,
                             int* cost) {
  clear_error();
  if (!s || !m || !cost) { set_error("phikron_setup_quadrature: NULL output"); return PHIKRON_EINVAL; }
  return planner::setup_quadrature(eps, p, alpha, beta, rule, s, m, cost);
}

int phikron_selector_features(int dims, const int* n, const double* tau_norm_inf, int l_max, double tol,
                              float* out8) {
  clear_error();
  if (dims < 1 || dims > 3 || !n || !tau_norm_inf || !out8 || l_max < 0 || !(tol > 0.0)) {
    set_error("phikron_selector_features: bad arguments");
    return PHIKRON_EINVAL;
  }
  selector_features(dims, n, tau_norm_inf, l_max, tol, out8);
  return PHIKRON_OK;
}

int phikron_gauss_legendre(int m, double* x, double* w) {
  clear_error();
  return planner::gauss_legendre(m, x, w);
}

int phikron_clenshaw_curtis(int n, double* x, double* w) {
  clear_error();
  return planner::clenshaw_curtis(n, x, w);
}

size_t phikron_expm_workspace_bytes(int count, int n) { return expm_workspace_bytes(count, n); }

int phikron_expm_batched(int count, int n, const double* A, const double* scale,
                         const double* norms1, double* E, void* workspace, void* stream) {
  clear_error();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<double> own;
  if (!norms1 && count > 0) {
    // ||A[b]||_1 (largest absolute column sum) from a host copy of the matrices: synchronous
    if (n < 1 || !A) {
      set_error("phikron_expm_batched: bad arguments");
      return PHIKRON_EINVAL;
    }
    const size_t nn = (size_t)n * n;
    std::vector<double> h(nn * count);
    PK_TRY_CUDA(cudaMemcpyAsync(h.data(), A, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
    PK_TRY_CUDA(cudaStreamSynchronize(st));
    own.assign(count, 0.0);
    std::vector<double> col(n);
    for (int b = 0; b < count; ++b) {
      std::fill(col.begin(), col.end(), 0.0);
      for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) col[k] += std::fabs(h[nn * b + (size_t)i * n + k]);
      own[b] = *std::max_element(col.begin(), col.end());
    }
    norms1 = own.data();
  }
  const size_t mats = sizeof(double) * (size_t)n * n * (size_t)std::max(count, 0);
  const chk::Range r[3] = {{A, mats}, {E, mats}, {workspace, expm_workspace_bytes(count, n)}};
  chk::CallScope cs(st, r, 3);
  PK_RET(cs.rc);
  return expm_batched(count, n, A, scale, norms1, E, workspace, st);
}

int phikron_kron_apply_f64(int dims, const int* n, const double* const* E, const double* V,
                           double* Out, double* work, void* stream) {
  clear_error();
  if (dims < 1 || dims > PHIKRON_MAX_DIMS || !n || !E || !V || !Out || !work) {
    set_error("phikron_kron_apply_f64: bad arguments");
    return PHIKRON_EINVAL;
  }
  long long N = 1;
  for (int d = 0; d < dims; ++d) {
    if (n[d] < 1 || !E[d]) {
      set_error("phikron_kron_apply_f64: bad size or matrix pointer");
      return PHIKRON_EINVAL;
    }
    N *= n[d];
  }
  // a mode product reads its whole input while it writes its output: V, Out and work must be
  // three separate ranges of N float64 (work is unused for one factor)
  if (ranges_overlap(V, Out, N) || (dims > 1 && (ranges_overlap(V, work, N) || ranges_overlap(Out, work, N)))) {
    set_error("phikron_kron_apply_f64: V, Out and work must not overlap");
    return PHIKRON_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  chk::Range r[PHIKRON_MAX_DIMS + 3];
  for (int d = 0; d < dims; ++d) r[d] = {E[d], sizeof(double) * (size_t)n[d] * n[d]};
  r[dims] = {V, sizeof(double) * (size_t)N};
  r[dims + 1] = {Out, sizeof(double) * (size_t)N};
  r[dims + 2] = {work, sizeof(double) * (size_t)N};
  chk::CallScope cs(st, r, dims + 3);
  PK_RET(cs.rc);
  const double* cur = V;
  for (int d = 0; d < dims; ++d) {
    long long B0 = 1, R = 1;
    for (int q = 0; q < d; ++q) B0 *= n[q];
    for (int q = d + 1; q < dims; ++q) R *= n[q];
    // ping-pong so that the last mode lands in Out: dims odd -> Out, work, Out ; even -> work, Out
    double* dst = (((dims - 1 - d) % 2) == 0) ? Out : work;
    PK_RET(mode_product_f64(cur, 0, dst, 0, E[d], 0, 1, B0, n[d], R, st));
    cur = dst;
  }
  return PHIKRON_OK;
}

}  // extern "C"
