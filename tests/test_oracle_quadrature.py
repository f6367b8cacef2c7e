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
