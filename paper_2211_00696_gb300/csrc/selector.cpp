// Measured error criterion and cost-minimising (s, m) search for the learned selector.
//
// For a symmetric A the error of the method in the 2-norm is the largest scalar error over
// the spectrum: ||phi_j(M)v - Phi_j(M)v||_2 <= max_{z in spec(M)} |phi_j(z) - Phi_j(z)| ||v||_2,
// where Phi_j is the method applied to the scalar z: Gauss-Legendre quadrature of Eq. (3) at
// 2^{-s} z (Algorithm 1) followed by s steps of the scalar modified squaring recurrence
// (Eq. (29)).  The criterion samples z over an interval [zlo, zhi] that encloses spec(M)
// (a Gershgorin bound at plan time) and takes the maximum over j = 1..p.  The search mirrors
// Algorithm 5 with this criterion in place of Theorem 3.2's bound: for each s the smallest m
// (2..32) meeting tol, cost m + s*p, scanning every s downward from a start above
// log2 ||M|| (Algorithm 5's early stop assumes a cost convex in s; with this criterion the
// cost can plateau, so the whole range is scanned).  These labels train the selector network.
#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

#include "common.h"

namespace phikron {
namespace selector {

namespace {

const double* inv_factorials() {
  static const std::vector<double> t = [] {
    std::vector<double> v(128);
    v[0] = 1.0;
    for (int k = 1; k < 128; ++k) v[k] = v[k - 1] / k;
    return v;
  }();
  return t.data();
}

// phi_j(z) for real z, j = 0..jmax (Taylor series for |z| <= jmax + 1, else the recurrence
// phi_j = (phi_{j-1} - 1/(j-1)!)/z read from phi_0 = e^z)
void phi_all(double z, int jmax, double* out) {
  const double* invf = inv_factorials();
  if (std::fabs(z) <= jmax + 1.0) {
    const int K = 60 + 2 * jmax;
    for (int j = 0; j <= jmax; ++j) {
      double acc = 0.0;
      for (int k = K; k >= 0; --k) acc = acc * z + invf[k + j];
      out[j] = acc;
    }
    return;
  }
  out[0] = std::exp(z);
  for (int j = 1; j <= jmax; ++j) out[j] = (out[j - 1] - invf[j - 1]) / z;
}

}  // namespace

// Largest error over the sample points of the scalar method (s, m) for phi_1..phi_p.
double criterion(double zlo, double zhi, int p, int s, int m, int npts) {
  std::vector<double> x(m), w(m);
  planner::gauss_legendre(m, x.data(), w.data());
  std::vector<double> inv_fact(p + 1);
  inv_fact[0] = 1.0;
  for (int j = 1; j <= p; ++j) inv_fact[j] = inv_fact[j - 1] / j;
  double worst = 0.0;
  std::vector<double> y(p + 1), yn(p + 1), ex(p + 2);
  for (int q = 0; q < npts; ++q) {
    // Chebyshev-distributed samples (dense near the interval ends) plus both end points
    const double t = (npts == 1) ? 0.0 : std::cos(M_PI * q / (npts - 1));
    const double z = 0.5 * (zlo + zhi) + 0.5 * (zhi - zlo) * t;
    const double zs = std::ldexp(z, -s);
    for (int j = 1; j <= p; ++j) y[j] = 0.0;
    for (int k = 0; k < m; ++k) {
      const double e = std::exp((1.0 - x[k]) * zs);
      double xp = 1.0;  // x_k^{j-1}
      for (int j = 1; j <= p; ++j) {
        y[j] += w[k] * xp * inv_fact[j - 1] * e;
        xp *= x[k];
      }
    }
    for (int t2 = 0; t2 < s; ++t2) {
      const double g = std::exp(std::ldexp(z, t2 - s));
      for (int i = 1; i <= p; ++i) {
        double acc = g * y[i];
        for (int j = 1; j <= i; ++j) acc += y[j] * inv_fact[i - j];
        yn[i] = std::ldexp(acc, -i);
      }
      for (int i = 1; i <= p; ++i) y[i] = yn[i];
    }
    phi_all(z, p, ex.data());
    for (int j = 1; j <= p; ++j) worst = std::max(worst, std::fabs(y[j] - ex[j]));
  }
  return worst;
}

int search(double zlo, double zhi, int p, double tol, int npts, int* s_out, int* m_out, int* cost_out) {
  const double a = std::max(std::fabs(zlo), std::fabs(zhi));
  int smax = (a > 0.0) ? (int)std::ceil(std::log2(a)) + 2 : 0;
  smax = std::max(0, std::min(20, smax));
  int best_cost = 1 << 30, bs = -1, bm = -1;
  for (int s = smax; s >= 0; --s) {
    // smallest m in 2..32 meeting tol (the criterion decreases with m)
    int lo = 2, hi = 32;
    if (criterion(zlo, zhi, p, s, hi, npts) > tol) {
      if (bs >= 0) break;  // cost can only grow further down in s
      continue;
    }
    while (lo < hi) {
      const int mid = (lo + hi) / 2;
      if (criterion(zlo, zhi, p, s, mid, npts) <= tol) hi = mid; else lo = mid + 1;
    }
    const int cost = lo + s * p;
    if (cost < best_cost) {  // full scan: the cost need not be convex in s (it can plateau)
      best_cost = cost;
      bs = s;
      bm = lo;
    }
  }
  if (bs < 0) {
    set_error("selector search: no (s, m) with s <= 20, m <= 32 meets the tolerance");
    return PHIKRON_ENOTCONVERGED;
  }
  *s_out = bs;
  *m_out = bm;
  *cost_out = best_cost;
  return PHIKRON_OK;
}

}  // namespace selector
}  // namespace phikron

using namespace phikron;

extern "C" {

int phikron_selector_criterion(double zlo, double zhi, int p, int s, int m, int npts, double* err) {
  clear_error();
  if (!err || p < 1 || p > 20 || s < 0 || s > 60 || m < 1 || m > 256 || npts < 1 || !(zlo <= zhi) ||
      zhi > 0.0) {
    set_error("phikron_selector_criterion: bad arguments (need zlo <= zhi <= 0, 1 <= p <= 20)");
    return PHIKRON_EINVAL;
  }
  *err = selector::criterion(zlo, zhi, p, s, m, npts);
  return PHIKRON_OK;
}

int phikron_selector_search(int count, const double* zlo, const double* zhi, const int* p, const double* tol,
                            int npts, int nthreads, int* s_out, int* m_out, int* cost_out) {
  clear_error();
  if (count < 0 || !zlo || !zhi || !p || !tol || !s_out || !m_out || !cost_out || npts < 2) {
    set_error("phikron_selector_search: bad arguments");
    return PHIKRON_EINVAL;
  }
  for (int i = 0; i < count; ++i) {
    if (!(zlo[i] <= zhi[i]) || zhi[i] > 0.0 || p[i] < 1 || p[i] > 20 || !(tol[i] > 0.0)) {
      set_error("phikron_selector_search: sample with bad interval, order or tolerance");
      return PHIKRON_EINVAL;
    }
  }
  if (nthreads < 1) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());
  nthreads = std::min(nthreads, std::max(1, count));
  std::vector<int> rc(nthreads, PHIKRON_OK);
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t) {
    th.emplace_back([&, t]() {
      for (int i = t; i < count; i += nthreads) {
        const int r = selector::search(zlo[i], zhi[i], p[i], tol[i], npts, &s_out[i], &m_out[i], &cost_out[i]);
        if (r != PHIKRON_OK) {
          s_out[i] = m_out[i] = cost_out[i] = -1;
          rc[t] = r;
        }
      }
    });
  }
  for (auto& x : th) x.join();
  for (int r : rc)
    if (r != PHIKRON_OK) {
      set_error("phikron_selector_search: some samples have no admissible (s, m) (marked -1)");
      return r;
    }
  return PHIKRON_OK;
}

}  // extern "C"
