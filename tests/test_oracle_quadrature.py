"""Pins for the oracle's restatement of Algorithms 1 and 6 against the plain definition."""
import numpy as np
import pytest

import workloads as W
from oracle import phi as P
from oracle import planner as PL
from oracle import quadrature as Q


def test_alg6_matches_O1_laplace2d_planned():
    prob = W.laplace2d(n=32, tau=1e-3, l_max=3, tol=1e-12)
    v = prob.vector()
    exact = P.phi_dense(prob.factors, prob.tau, v, prob.l_max)
    got, st = Q.alg6_phiquadmv(prob.factors, prob.tau, v, prob.l_max, prob.tol, return_stages=True)
    assert st["s"] >= 1
    for l in range(prob.l_max + 1):
        assert P.rel_err_2(got[l], exact[l]) <= 1e-12


@pytest.mark.parametrize("s", [0, 2, 4])
def test_alg6_matches_O1_nonsymmetric_3d_forced_scaling(s):
    fac = [W.convdiff_factor(n) for n in (6, 5, 7)]
    tau, p = 1e-2, 3
    v = W.uniform_vector((6, 5, 7), 1)
    exact = P.phi_dense(fac, tau, v, p)
    got, st = Q.alg6_phiquadmv(fac, tau, v, p, 1e-12, s=s, m=12, return_stages=True)
    for l in range(p + 1):
        assert P.rel_err_2(got[l], exact[l]) <= 2e-13
    scaled = P.phi_dense(fac, tau / 2 ** s, v, p)
    for j in range(1, p + 1):
        assert P.rel_err_2(st["scaled"][j - 1], scaled[j]) <= 2e-13


def test_alg6_cc_rule_matches_O1():
    fac = [W.laplacian_factor(9), W.convdiff_factor(8)]
    tau, p = 2e-3, 2
    v = W.uniform_vector((9, 8), 2)
    exact = P.phi_dense(fac, tau, v, p)
    got = Q.alg6_phiquadmv(fac, tau, v, p, 1e-12, s=2, m=17, rule=PL.CC)
    for l in range(p + 1):
        assert P.rel_err_2(got[l], exact[l]) <= 1e-12


# ----------------------------------------------------------------------------- Algorithm 2

def test_clenshaw_curtis_rules_are_nested():
    """Algorithm 2 reuses the integrand at the old nodes: the even points of the (2n+1)-point
    rule are the (n+1)-point rule."""
    from oracle import planner as PL
    for n in (3, 6, 12, 24):
        x2, _ = PL.clenshaw_curtis_01(2 * n)
        x1, _ = PL.clenshaw_curtis_01(n)
        assert np.array_equal(x2[::2], x1)


@pytest.mark.parametrize("tol", [1e-6, 1e-10, 1e-13])
def test_alg2_adaptive_matches_definition(tol):
    fac = [W.convdiff_factor(5), W.laplacian_factor(4, 0.8), W.convdiff_factor(3)]
    tau, p = 2e-2, 3
    v = np.random.default_rng(4).uniform(-1, 1, 60)
    out, st = Q.alg6_phiquadmv(fac, tau, v, p, tol, rule="cc_adaptive", return_stages=True)
    exact = P.phi_dense(fac, tau, v, p)
    assert st["err"] <= tol and st["nodes"] in (13, 25, 49, 97, 193, 385)
    for l in range(p + 1):
        assert P.rel_err_2(out[l], exact[l]) <= 5 * tol + 1e-14, (l, st)


def test_alg2_diagonal_operator_gives_scalar_phi():
    """Diagonal factors: y_j is phi_j of the diagonal entries (closed form via the scalar
    recurrence), so the adaptive rule's result must meet its tolerance entrywise."""
    d = [np.diag([-0.3, -2.0, -5.5]), np.diag([-0.1, -1.7])]
    v = np.array([0.3, -1.0, 2.0, 0.5, -0.7, 1.1])
    y, nodes, err = Q.alg2_adaptive_cc(d, v, 3, 1e-12)
    z = (np.diag(d[0])[:, None] + np.diag(d[1])[None, :]).ravel()
    for j in range(1, 4):
        ref = P.phi_scalar(j, z) * v
        assert np.max(np.abs(y[j - 1] - ref)) <= 1e-11 * np.max(np.abs(ref)), j
    assert err <= 1e-12


def test_remark_combo_equals_sum_of_phi_actions():
    """The Remark's single quadrature of sum_j phi_j(M) b_j agrees with the separate
    phi-actions of the dense definition (Gauss rule, s = 0, small tau||A||)."""
    from oracle import planner as PL
    fac = [W.convdiff_factor(5), W.laplacian_factor(4, 0.5)]
    tau, p = 4e-3, 3
    rng = np.random.default_rng(6)
    B = [rng.uniform(-1, 1, 20) for _ in range(p)]
    x, w = PL.gauss_legendre_01(10)
    got = Q.remark_combo(fac, tau, B, x, w)
    ref = sum(P.phi_dense(fac, tau, B[j - 1], p)[j] for j in range(1, p + 1))
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
