"""Pins for the oracle's exponential Runge-Kutta steps (Eq. (RK), Table RK), on the CPU:
exactness for f = 0 and f = const (the exact solution of the linear problem), and the orders
1, 2, 3 against an independent stiff ODE solver."""
import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

import workloads as W
from oracle import erk as E
from oracle import phi as P


def _small_problem():
    fac = [W.convdiff_factor(4), W.laplacian_factor(3, 0.7)]
    return fac, P.kron_sum_dense(fac)


@pytest.mark.parametrize("name", ["euler", "rk2", "rk3"])
def test_linear_problem_is_propagated_exactly(name):
    fac, A = _small_problem()
    rng = np.random.default_rng(1)
    u = rng.uniform(-1, 1, A.shape[0])
    c = rng.uniform(-1, 1, A.shape[0])
    tau = 0.05
    phi = lambda t, v, p: P.phi_dense(fac, t, v, p)
    A_apply = lambda x: E.kron_sum_apply(fac, x)
    tab = E.TABLEAUS[name]()
    # f = 0: u+ = e^{-tau A} u
    got = E.step(tab, u, tau, lambda x: np.zeros_like(x), A_apply, phi)
    ref = scipy.linalg.expm(-tau * A) @ u
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    # f = c: u+ = e^{-tau A} u + tau phi_1(-tau A) c, with phi_1 from A^{-1}(I - e^{-tau A}) / tau
    got = E.step(tab, u, tau, lambda x: c, A_apply, phi)
    ref = scipy.linalg.expm(-tau * A) @ u + np.linalg.solve(A, c - scipy.linalg.expm(-tau * A) @ c)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_kron_sum_apply_matches_assembled_matrix():
    fac = [W.convdiff_factor(5), W.laplacian_factor(3), W.periodic_diffusion_factor(4, 0.3)]
    u = np.random.default_rng(2).standard_normal(60)
    assert np.allclose(E.kron_sum_apply(fac, u), P.kron_sum_dense(fac) @ u, rtol=1e-14, atol=1e-12)


@pytest.mark.parametrize("name,order", [("euler", 1), ("rk2", 2), ("rk3", 3)])
def test_observed_order_against_stiff_solver(name, order):
    """Allen-Cahn on an 8 x 7 Dirichlet grid (coefficient 0.1, ||A||_2 = 56), smooth initial
    data, T = 1, reference from scipy's Radau at rtol 1e-13: the error ratio between tau and
    tau/2 approaches 2^order (the stiff orders of the three methods)."""
    n1, n2 = 8, 7
    fac = [W.laplacian_factor(n1, 0.1), W.laplacian_factor(n2, 0.1)]
    A = P.kron_sum_dense(fac)
    x = np.arange(1, n1 + 1) / (n1 + 1)
    y = np.arange(1, n2 + 1) / (n2 + 1)
    u0 = (0.9 * np.outer(np.sin(np.pi * x), np.sin(np.pi * y))
          + 0.3 * np.outer(np.sin(2 * np.pi * x), np.sin(3 * np.pi * y))).ravel()
    T = 1.0
    sol = scipy.integrate.solve_ivp(lambda t, v: -A @ v + E.allen_cahn(v), (0, T), u0, method="Radau",
                                    rtol=1e-13, atol=1e-14, jac=lambda t, v: -A + np.diag(1 - 3 * v * v))
    ref = sol.y[:, -1]
    phi = lambda t, v, p: P.phi_dense(fac, t, v, p)
    A_apply = lambda v: E.kron_sum_apply(fac, v)
    errs = []
    for nsteps in (16, 32, 64):
        got = E.integrate(E.TABLEAUS[name](), u0, T / nsteps, nsteps, E.allen_cahn, A_apply, phi)
        errs.append(np.max(np.abs(got - ref)))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) >= order - 0.15, (errs, rates)
    assert max(rates) <= order + 0.3, (errs, rates)
