"""Quadrature rules and the a-priori planner of Sec. 3.2-3.3.  Test infrastructure only.

* ``gauss_legendre_01`` / ``clenshaw_curtis_01`` -- the (n+1)-point rules on [0, 1]
  (Sec. 3.1, Eq. (10)); Gauss-Legendre from numpy's ``leggauss`` (library step),
  Clenshaw-Curtis from its explicit cosine-sum weights.
* ``log_bound``   -- log of the Theorem 3.2 bound, Eqs. (14)-(16), for a given rho.
* ``quaderr``     -- Algorithm 3: max over q = 1..p of the bound minimised over the real
                     roots rho > 1 of the quartic of Eqs. (17)-(18) (numpy.roots).
* ``quadnodes``   -- Algorithm 4: start at n = 2 (Gauss) / 4 (CC), double while the
                     bound exceeds eps, then the root of quaderr(n) - eps on [n/2, n]
                     over continuous n, rounded up.
* ``setup_quadrature`` -- Algorithm 5: scan l = ceil(log2 alpha) .. 0, cost
                     C = (n+1) + l*p (c1 = 0, c2 = 1, Sec. 4), stop at the first l whose
                     cost does not improve.
* ``corollary_bound`` -- the closed forms of Corollary 3.3, Eqs. (19)-(20).

Readings of the paper taken here (each is also listed in the design notes):
  - The node count is n+1 and Tables 2 and 4 print it (n-bar) with C-bar = (n+1) + l*p.
  - Algorithm 3 works in logarithms (Remark 3.3).  Among the real roots > 1 of the
    quartic the one giving the smallest bound is used (Algorithm 3, step 2).
  - Algorithm 4: if the starting n already meets eps it is returned as is.
  - Algorithm 5: l_max = ceil(log2 alpha) clamped at 0; a tie in cost stops the scan.
  - beta = 1 with eps = tol makes the tolerance relative to ||v||_inf.
Parity: pinned by Tables 2 and 4 (exact integers), by root-existence and monotonicity
properties, and by the quadrature error it predicts (tests/test_oracle_planner.py).
"""
from __future__ import annotations

import math

import numpy as np

GAUSS = "gauss"
CC = "cc"
LOG_144_35 = math.log(144.0 / 35.0)


# ----------------------------------------------------------------------------- rules

def gauss_legendre_01(m: int):
    """m-point Gauss-Legendre nodes/weights on [0,1] (numpy's leggauss mapped affinely)."""
    t, w = np.polynomial.legendre.leggauss(m)
    return 0.5 * (t + 1.0), 0.5 * w


def clenshaw_curtis_01(n: int):
    """(n+1)-point Clenshaw-Curtis rule on [0,1], nodes x_j = (1 - cos(j pi/n))/2.

    Weights on [-1,1]: w_j = (c_j/n)(1 - sum_{k=1}^{floor(n/2)} b_k cos(2 k j pi/n)/(4k^2-1)),
    c_0 = c_n = 1, c_j = 2 otherwise; b_k = 1 if k = n/2 else 2.  Halved for [0,1].
    """
    j = np.arange(n + 1)
    theta = j * np.pi / n
    x = 0.5 * (1.0 - np.cos(theta))
    w = np.zeros(n + 1)
    for jj in range(n + 1):
        s = 0.0
        for k in range(1, n // 2 + 1):
            b = 1.0 if 2 * k == n else 2.0
            s += b * math.cos(2 * k * theta[jj]) / (4 * k * k - 1)
        c = 1.0 if jj in (0, n) else 2.0
        w[jj] = c / n * (1.0 - s)
    return x, 0.5 * w


# ----------------------------------------------------------------------------- Theorem 3.2

def quartic_coeffs(n: float, p: int, alpha: float, rule: str = GAUSS):
    """(a3, a2, a1) of Eq. (18) for the monic quartic rho^4 + a3 rho^3 + a2 rho^2 + a1 rho + 1."""
    if rule == GAUSS:
        a3 = -4.0 / alpha * (2.0 * (n + 1.0) - p)
        a1 = 4.0 / alpha * (2.0 * n + p)
    else:
        a3 = -4.0 / alpha * (n + 1.0 - p)
        a1 = 4.0 / alpha * (n - 1.0 + p)
    a2 = -(2.0 + 8.0 * p / alpha)
    return a3, a2, a1


def log_bound(rho: float, n: float, p: int, alpha: float, beta: float, rule: str = GAUSS) -> float:
    """log of Eq. (15) (Gauss) or Eq. (14) (CC) with M(rho) of Eq. (16), for phi_{p+1}."""
    g = (rho + 1.0) ** 2 / (2.0 * rho)
    logM = p * math.log(g) - (p + 1) * math.log(2.0) - math.lgamma(p + 1) + 0.5 * g * alpha + math.log(beta)
    if rule == GAUSS:
        pw = -2.0 * n * math.log(rho)
    else:
        pw = (1.0 - n) * math.log(rho)
    return LOG_144_35 + logM + pw - math.log(rho * rho - 1.0)


def real_roots_above_one(coeffs):
    r = np.roots(coeffs)
    out = []
    for z in r:
        if abs(z.imag) <= 1e-9 * abs(z) and z.real > 1.0:
            out.append(float(z.real))
    return out


def log_quaderr(n: float, p: int, alpha: float, beta: float, rule: str = GAUSS) -> float:
    """Algorithm 3 in logarithms: max_{q=1..p} min over admissible roots of the bound."""
    E = -math.inf
    nn = n
    if rule == CC and abs(n - round(n)) < 1e-12 and int(round(n)) % 2 == 0:
        nn = n + 1.0  # Theorem 3.2: for even n the CC bound may use n+1
    for q in range(1, p + 1):
        pt = q - 1
        a3, a2, a1 = quartic_coeffs(nn, pt, alpha, rule)
        roots = real_roots_above_one([1.0, a3, a2, a1, 1.0])
        if not roots:
            raise ArithmeticError("quartic of Eq. (17) has no real root > 1")
        Ebar = min(log_bound(r, nn, pt, alpha, beta, rule) for r in roots)
        E = max(E, Ebar)
    return E


def quaderr(n, p, alpha, beta, rule=GAUSS) -> float:
    return math.exp(log_quaderr(n, p, alpha, beta, rule))


def quadnodes(eps: float, p: int, alpha: float, beta: float, rule: str = GAUSS) -> int:
    """Algorithm 4: returns n (the rule then has n+1 nodes)."""
    log_eps = math.log(eps)
    n = 2 if rule == GAUSS else 4
    if log_quaderr(n, p, alpha, beta, rule) <= log_eps:
        return n
    while log_quaderr(n, p, alpha, beta, rule) > log_eps:
        n *= 2
    lo, hi = n / 2.0, float(n)
    # bisection on h(n) = log quaderr(n) - log eps, h(lo) > 0 >= h(hi)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if log_quaderr(mid, p, alpha, beta, rule) > log_eps:
            lo = mid
        else:
            hi = mid
        if hi - lo <= 1e-12 * hi:
            break
    return int(math.ceil(hi))


def setup_quadrature(eps: float, p: int, alpha: float, beta: float = 1.0, rule: str = GAUSS):
    """Algorithm 5: returns (l_bar, m_bar = n_bar + 1 nodes, C_bar = m_bar + l_bar*p)."""
    lmax = max(0, int(math.ceil(math.log2(alpha)))) if alpha > 0 else 0
    best = (None, None, math.inf)
    for l in range(lmax, -1, -1):
        n = quadnodes(eps, p, alpha / 2.0 ** l, beta, rule)
        C = (n + 1) + l * p
        if C < best[2]:
            best = (l, n + 1, C)
        else:
            break
    return best


def corollary_bound(n: int, p: int, alpha: float, beta: float, rule: str = GAUSS) -> float:
    """Corollary 3.3 closed forms, Eqs. (19)-(20), for phi_{p+1} with n+1 nodes.

    Valid for n >= (1+sqrt 2)/4 * alpha + p/2 (Gauss), n >= (1+sqrt 2)/2 * alpha + p and
    n even (CC; odd n uses n-1).  Returns +inf outside that range.
    """
    c = beta / (2.0 ** (p + 1) * math.factorial(p))
    if rule == GAUSS:
        if n < max(2, (1 + math.sqrt(2)) / 4 * alpha + p / 2):
            return math.inf
        k = 2 * n - p
    else:
        if n % 2 == 1:
            n -= 1
        if n < max(4, (1 + math.sqrt(2)) / 2 * alpha + p):
            return math.inf
        k = n - p
    return c * (k / (math.e / 2 * alpha)) ** (-k)


def alpha_inf(factors, tau: float) -> float:
    """alpha = tau * sum_d ||A^d||_inf, the upper bound of Eq. (31)."""
    return tau * sum(float(np.max(np.sum(np.abs(a), axis=1))) for a in factors)
