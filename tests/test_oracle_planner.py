"""Pins for the oracle's planner (Algorithms 3-5) and quadrature rules -- CPU only.

Exact-integer pins come from the paper's Tables 2 and 4 (tests/golden).  The bound
itself is pinned by the quadrature error it must dominate (Theorem 3.2, Corollary 3.3),
computed against the plain definition (O1).
"""
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import phi as P
from oracle import planner as PL
from oracle import quadrature as Q

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([float(t) for t in line.split()])
    return rows


@pytest.mark.parametrize("table", ["table2_points_laplace.txt", "table4_points_advdiff.txt"])
def test_setup_quadrature_reproduces_paper_tables(table):
    for size, alpha, g_n, g_C, g_l, cc_n, cc_C, cc_l in _table(table):
        l, m, C = PL.setup_quadrature(1e-14, 20, alpha, 1.0, PL.GAUSS)
        assert (l, m, C) == (int(g_l), int(g_n), int(g_C)), (alpha, l, m, C)
        l_cc, _, _ = PL.setup_quadrature(1e-14, 20, alpha, 1.0, PL.CC)
        assert l_cc == int(cc_l)


def test_quartic_has_root_above_one_always():
    """Sec. 3.2 proof (Descartes' rule on Q(x) = P(1+x)): a real root > 1 exists."""
    for rule in (PL.GAUSS, PL.CC):
        for n in (2, 3, 5, 8, 17, 40, 100, 2.5, 7.25):
            for p in range(0, 21, 4):
                for alpha in (1e-3, 0.1, 1.0, 5.0, 50.0, 1e3, 1e5):
                    a3, a2, a1 = PL.quartic_coeffs(n, p, alpha, rule)
                    assert PL.real_roots_above_one([1.0, a3, a2, a1, 1.0])


def test_quartic_root_is_stationary_point_of_log_bound():
    """The roots of Eq. (17) are the critical points of the log-bound minimised in the proof."""
    n, p, alpha = 9.0, 3, 6.0
    a3, a2, a1 = PL.quartic_coeffs(n, p, alpha)
    for r in PL.real_roots_above_one([1.0, a3, a2, a1, 1.0]):
        h = 1e-6 * r
        d = (PL.log_bound(r + h, n, p, alpha, 1.0) - PL.log_bound(r - h, n, p, alpha, 1.0)) / (2 * h)
        assert abs(d) < 1e-6


def test_quaderr_decreases_in_n_and_quadnodes_is_minimal():
    for p, alpha, eps in [(3, 8.7, 1e-10), (3, 27.7 / 8, 1e-10), (20, 3.0, 1e-14), (1, 0.5, 1e-6)]:
        prev = math.inf
        for n in range(2, 60):
            e = PL.quaderr(n, p, alpha, 1.0)
            assert e < prev
            prev = e
        n = PL.quadnodes(eps, p, alpha, 1.0)
        assert PL.quaderr(n, p, alpha, 1.0) <= eps
        if n > 2:
            assert PL.quaderr(n - 1, p, alpha, 1.0) > eps


def test_gauss_legendre_exact_for_degree_2m_minus_1():
    for m in (1, 2, 5, 9, 16, 33):
        x, w = PL.gauss_legendre_01(m)
        for k in range(2 * m):
            assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) <= 1e-14
        assert np.all((x > 0) & (x < 1))


def test_clenshaw_curtis_exact_for_degree_n():
    for n in (2, 4, 6, 12, 24, 48):
        x, w = PL.clenshaw_curtis_01(n)
        for k in range(n + 1 + (n % 2 == 0)):
            assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) <= 1e-14


def _quad_error(shape, tau, p, m, rule):
    fac = [W.laplacian_factor(n) for n in shape]
    v = W.uniform_vector(shape, 21)
    exact = P.phi_dense(fac, tau, v, p)
    Ms = [-tau * a for a in fac]
    if rule == PL.GAUSS:
        x, w = PL.gauss_legendre_01(m)
    else:
        x, w = PL.clenshaw_curtis_01(m - 1)
    ys = Q.alg1_fixed(Ms, v, p, x, w)
    err = max(np.max(np.abs(ys[j - 1] - exact[j])) for j in range(1, p + 1))
    alpha = PL.alpha_inf(fac, tau)
    return err, alpha, float(np.max(np.abs(v))), exact, ys


def test_theorem32_bound_dominates_quadrature_error():
    shape, tau, p = (10, 12), 3e-3, 3
    for m in range(3, 13):
        err, alpha, beta, _, _ = _quad_error(shape, tau, p, m, PL.GAUSS)
        bound = PL.quaderr(m - 1, p, alpha, beta, PL.GAUSS)
        assert err <= bound * (1 + 1e-9) + 1e-14, (m, err, bound)
    for m in range(5, 16):
        err, alpha, beta, _, _ = _quad_error(shape, tau, p, m, PL.CC)
        bound = PL.quaderr(m - 1, p, alpha, beta, PL.CC)
        assert err <= bound * (1 + 1e-9) + 1e-14, (m, err, bound)


def test_corollary33_bound_dominates_and_is_supergeometric():
    shape, tau, p = (10, 12), 3e-3, 2
    errs = []
    for m in range(3, 11):
        err, alpha, beta, _, _ = _quad_error(shape, tau, p, m, PL.GAUSS)
        errs.append(err)
        cb = max(PL.corollary_bound(m - 1, q - 1, alpha, beta, PL.GAUSS) for q in range(1, p + 1))
        assert err <= cb * (1 + 1e-9) + 1e-14
    # supergeometric: successive error ratios keep shrinking while above roundoff
    ratios = [errs[i + 1] / errs[i] for i in range(len(errs) - 1) if errs[i + 1] > 1e-14]
    assert all(ratios[i + 1] < ratios[i] for i in range(len(ratios) - 1))


def test_gauss_and_cc_agree():
    shape, tau, p = (8, 9), 2e-3, 3
    _, _, _, exact, yg = _quad_error(shape, tau, p, 14, PL.GAUSS)
    _, _, _, _, yc = _quad_error(shape, tau, p, 25, PL.CC)
    for j in range(p):
        assert P.rel_err_2(yg[j], yc[j]) <= 1e-12


def test_twenty_one_nodes_claim_sec33():
    """Scaling with l = log2(e alpha/2) makes ||2^-l A|| = 2/e; 21 nodes then suffice for
    error below 1e-20 ||b|| for p <= 20 (Sec. 3.3, Eq. (30))."""
    for p in range(0, 21):
        simplified = 1.0 / (2 ** (p + 1) * math.factorial(p)) * (2 * 20 - p) ** (-(2 * 20 - p))
        assert simplified < 1e-20
    assert PL.quaderr(20, 20, 2.0 / math.e, 1.0) < 1e-20


def test_alpha_inf_is_the_max_row_sum_on_nonsymmetric_factors():
    """Eq. (31) sums the infinity norms (maximum absolute ROW sum) of the factors.  These factors
    are neither symmetric nor Toeplitz, so their row and column sums differ, and so do the max
    of row sums and the sum of all entries; the values are worked out by hand:
      A1 = [[1, -2], [0, 3]]            row sums 3, 3        -> 3   (column sums 1, 5 -> 5)
      A2 = [[0, 0, 4], [-1, 1, 0],
            [0.5, 0, 0]]                row sums 4, 2, 0.5   -> 4   (column sums 1.5, 1, 4)
      A3 = [[-7]]                                            -> 7
    alpha = tau * (3 + 4 + 7) = 14 tau."""
    A1 = np.array([[1.0, -2.0], [0.0, 3.0]])
    A2 = np.array([[0.0, 0.0, 4.0], [-1.0, 1.0, 0.0], [0.5, 0.0, 0.0]])
    A3 = np.array([[-7.0]])
    assert PL.alpha_inf([A1], 1.0) == 3.0
    assert PL.alpha_inf([A1.T], 1.0) == 5.0          # the transpose has the column sums as rows
    assert PL.alpha_inf([A2], 1.0) == 4.0
    assert PL.alpha_inf([A1, A2, A3], 0.25) == 0.25 * 14.0
    # a single row: the inf-norm is the sum of |entries| in it, not their max
    assert PL.alpha_inf([np.array([[2.0, -3.0], [0.0, 0.0]])], 1.0) == 5.0
