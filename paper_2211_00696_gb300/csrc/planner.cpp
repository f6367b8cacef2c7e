// Host planner (scalar work of Algorithm 6's first step): the a-priori quadrature bound of
// Theorem 3.2 (Sec. 3.2), Algorithms 3 (quaderr), 4 (quadnodes) and 5 (setup_quadrature),
// and the quadrature rules.  Pure C++, no CUDA.
//
// Readings of the paper implemented here:
//  * Work in logarithms of the bound (Remark 3.3).
//  * Algorithm 3: for q = 1..p use Eq. (18) with p := q-1, keep the real roots rho > 1 of the
//    quartic Eq. (17) (|Im rho| <= 1e-9 |rho|), take the smallest bound among them, and the
//    largest over q.  No admissible root => PHIKRON_ENOTCONVERGED (the proof of Theorem 3.2
//    guarantees one exists for n >= 2, alpha > 0).
//  * Algorithm 4: start at n = 2 (Gauss) or 4 (CC); a start that already meets eps is
//    returned as is; otherwise double n, then bisect the continuous root of
//    log quaderr(n) - log eps on [n/2, n] and round up.
//  * Algorithm 5: l_max = ceil(log2 alpha) (at least 0), cost C = (n+1) + l*p (c1 = 0,
//    c2 = 1 as in Sec. 4), stop at the first l whose cost does not improve.
//  * For CC and even n, Theorem 3.2 allows n+1 in place of n.
#include <cmath>
#include <complex>
#include <limits>

#include "common.h"

namespace phikron {
namespace planner {

namespace {

using cd = std::complex<double>;

// All four roots of z^4 + c3 z^3 + c2 z^2 + c1 z + c0 by the Aberth-Ehrlich simultaneous
// iteration (cubically convergent), each then polished by Newton steps.
bool quartic_roots(double c3, double c2, double c1, double c0, cd r[4]) {
  const double c[5] = {1.0, c3, c2, c1, c0};
  auto poly = [&](cd z) { return (((z + c3) * z + c2) * z + c1) * z + c0; };
  auto dpoly = [&](cd z) { return ((4.0 * z + 3.0 * c3) * z + 2.0 * c2) * z + c1; };
  double R = 0.0;
  for (int i = 1; i < 5; ++i) R = std::fmax(R, std::fabs(c[i]));
  R = 1.0 + R;  // Cauchy bound on |root|
  double rho0 = std::pow(std::fabs(c0), 0.25);
  double rad = std::fmin(R, std::fmax(rho0, 1e-3));
  for (int i = 0; i < 4; ++i) {
    double ang = 2.0 * M_PI * i / 4.0 + 0.4;
    r[i] = cd(rad * std::cos(ang), rad * std::sin(ang));
  }
  bool converged = false;
  for (int it = 0; it < 500 && !converged; ++it) {
    converged = true;
    for (int i = 0; i < 4; ++i) {
      cd p = poly(r[i]);
      cd dp = dpoly(r[i]);
      if (std::abs(p) == 0.0) continue;
      cd ratio = (std::abs(dp) > 0.0) ? p / dp : cd(1e-3, 1e-3);
      cd s(0.0, 0.0);
      for (int j = 0; j < 4; ++j)
        if (j != i) {
          cd dz = r[i] - r[j];
          if (std::abs(dz) > 0.0) s += 1.0 / dz;
        }
      cd denom = 1.0 - ratio * s;
      cd step = (std::abs(denom) > 0.0) ? ratio / denom : ratio;
      r[i] -= step;
      if (std::abs(step) > 1e-15 * std::fmax(1.0, std::abs(r[i]))) converged = false;
    }
  }
  for (int i = 0; i < 4; ++i) {
    for (int k = 0; k < 3; ++k) {
      cd dp = dpoly(r[i]);
      if (std::abs(dp) == 0.0) break;
      cd step = poly(r[i]) / dp;
      if (!(std::abs(step) < 1e-2 * std::fmax(1.0, std::abs(r[i])))) break;
      r[i] -= step;
    }
  }
  for (int i = 0; i < 4; ++i)
    if (!std::isfinite(r[i].real()) || !std::isfinite(r[i].imag())) return false;
  return true;
}

double log_bound(double rho, double n, int p, double alpha, double beta, int rule) {
  const double g = (rho + 1.0) * (rho + 1.0) / (2.0 * rho);
  const double logM = p * std::log(g) - (p + 1) * std::log(2.0) - std::lgamma(p + 1.0) +
                      0.5 * g * alpha + std::log(beta);
  const double pw = (rule == PHIKRON_QUAD_GAUSS) ? -2.0 * n * std::log(rho)
                                                 : (1.0 - n) * std::log(rho);
  return std::log(144.0 / 35.0) + logM + pw - std::log(rho * rho - 1.0);
}

}  // namespace

int log_quaderr(double n, int p, double alpha, double beta, int rule, double* out) {
  if (!(alpha > 0.0) || !(beta > 0.0) || !(n >= 1.0) || p < 1 || !std::isfinite(alpha)) {
    set_error("log_quaderr: need alpha > 0, beta > 0, n >= 1, p >= 1");
    return PHIKRON_EINVAL;
  }
  double nn = n;
  if (rule == PHIKRON_QUAD_CC && std::fabs(n - std::round(n)) < 1e-12 &&
      (static_cast<long long>(std::llround(n)) % 2 == 0))
    nn = n + 1.0;
  double E = -std::numeric_limits<double>::infinity();
  for (int q = 1; q <= p; ++q) {
    const int pt = q - 1;
    double a3, a1;
    if (rule == PHIKRON_QUAD_GAUSS) {
      a3 = -4.0 / alpha * (2.0 * (nn + 1.0) - pt);
      a1 = 4.0 / alpha * (2.0 * nn + pt);
    } else {
      a3 = -4.0 / alpha * (nn + 1.0 - pt);
      a1 = 4.0 / alpha * (nn - 1.0 + pt);
    }
    const double a2 = -(2.0 + 8.0 * pt / alpha);
    cd r[4];
    if (!quartic_roots(a3, a2, a1, 1.0, r)) {
      set_error("log_quaderr: quartic root iteration failed");
      return PHIKRON_ENOTCONVERGED;
    }
    double best = std::numeric_limits<double>::infinity();
    bool found = false;
    for (int i = 0; i < 4; ++i) {
      if (std::fabs(r[i].imag()) <= 1e-9 * std::abs(r[i]) && r[i].real() > 1.0) {
        const double lb = log_bound(r[i].real(), nn, pt, alpha, beta, rule);
        if (lb < best) best = lb;
        found = true;
      }
    }
    if (!found) {
      set_error("log_quaderr: the quartic of Theorem 3.2 has no real root > 1");
      return PHIKRON_ENOTCONVERGED;
    }
    if (best > E) E = best;
  }
  *out = E;
  return PHIKRON_OK;
}

int quadnodes(double eps, int p, double alpha, double beta, int rule, int* n_out) {
  if (!(eps > 0.0)) {
    set_error("quadnodes: eps must be > 0");
    return PHIKRON_EINVAL;
  }
  const double leps = std::log(eps);
  int n = (rule == PHIKRON_QUAD_GAUSS) ? 2 : 4;
  double E;
  PK_RET(log_quaderr(n, p, alpha, beta, rule, &E));
  if (E <= leps) {
    *n_out = n;
    return PHIKRON_OK;
  }
  while (E > leps) {
    if (n > (1 << 20)) {
      set_error("quadnodes: node count diverged");
      return PHIKRON_ENOTCONVERGED;
    }
    n *= 2;
    PK_RET(log_quaderr(n, p, alpha, beta, rule, &E));
  }
  double lo = 0.5 * n, hi = n;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    double Em;
    PK_RET(log_quaderr(mid, p, alpha, beta, rule, &Em));
    if (Em > leps)
      lo = mid;
    else
      hi = mid;
    if (hi - lo <= 1e-12 * hi) break;
  }
  *n_out = static_cast<int>(std::ceil(hi));
  return PHIKRON_OK;
}

int setup_quadrature(double eps, int p, double alpha, double beta, int rule, int* s, int* m,
                     int* cost) {
  if (!(alpha > 0.0) || !std::isfinite(alpha)) {
    set_error("setup_quadrature: alpha must be finite and > 0");
    return PHIKRON_EINVAL;
  }
  int lmax = static_cast<int>(std::ceil(std::log2(alpha)));
  if (lmax < 0) lmax = 0;
  long long bestC = std::numeric_limits<long long>::max();
  int bs = -1, bm = -1;
  for (int l = lmax; l >= 0; --l) {
    int n;
    PK_RET(quadnodes(eps, p, std::ldexp(alpha, -l), beta, rule, &n));
    const long long C = (long long)(n + 1) + (long long)l * p;
    if (C < bestC) {
      bestC = C;
      bs = l;
      bm = n + 1;
    } else {
      break;
    }
  }
  *s = bs;
  *m = bm;
  *cost = static_cast<int>(bestC);
  return PHIKRON_OK;
}

int gauss_legendre(int m, double* x, double* w) {
  if (m < 1 || m > 256 || !x || !w) {
    set_error("gauss_legendre: need 1 <= m <= 256 and non-null outputs");
    return PHIKRON_EINVAL;
  }
  // Roots t_i of P_m by Newton's method on the three-term recurrence, starting from the
  // asymptotic guess cos(pi (i - 1/4)/(m + 1/2)); weights 2 / ((1 - t^2) P_m'(t)^2).  The
  // recurrence runs in long double so the weights keep full double accuracy up to m = 256.
  typedef long double ld;
  auto legendre = [m](ld t, ld* pm, ld* pm1) {
    ld p0 = 1.0L, p1 = t;
    for (int k = 1; k < m; ++k) {
      const ld p2 = ((2.0L * k + 1.0L) * t * p1 - k * p0) / (k + 1.0L);
      p0 = p1;
      p1 = p2;
    }
    *pm = p1;
    *pm1 = p0;
  };
  for (int i = 0; i < m; ++i) {
    ld t = std::cos(M_PI * (i + 0.75) / (m + 0.5));
    ld pm, pm1, dp;
    for (int it = 0; it < 100; ++it) {
      legendre(t, &pm, &pm1);
      dp = m * (t * pm - pm1) / (t * t - 1.0L);
      const ld dt = pm / dp;
      t -= dt;
      if (std::fabs((double)dt) <= 1e-19 * std::fmax(1.0, std::fabs((double)t))) break;
    }
    legendre(t, &pm, &pm1);
    dp = m * (t * pm - pm1) / (t * t - 1.0L);
    // t decreases with i, so x = (1 - t)/2 increases
    x[i] = (double)(0.5L * (1.0L - t));
    w[i] = (double)(1.0L / ((1.0L - t) * (1.0L + t) * dp * dp));  // 2/(...) halved for [0,1]
  }
  return PHIKRON_OK;
}

int clenshaw_curtis(int n, double* x, double* w) {
  if (n < 1 || n > 512 || !x || !w) {
    set_error("clenshaw_curtis: need 1 <= n <= 512 and non-null outputs");
    return PHIKRON_EINVAL;
  }
  for (int j = 0; j <= n; ++j) {
    const double th = j * M_PI / n;
    x[j] = 0.5 * (1.0 - std::cos(th));
    double s = 0.0;
    for (int k = 1; 2 * k <= n; ++k) {
      const double b = (2 * k == n) ? 1.0 : 2.0;
      s += b * std::cos(2.0 * k * th) / (4.0 * k * k - 1.0);
    }
    const double c = (j == 0 || j == n) ? 1.0 : 2.0;
    w[j] = 0.5 * c / n * (1.0 - s);
  }
  return PHIKRON_OK;
}

}  // namespace planner
}  // namespace phikron
