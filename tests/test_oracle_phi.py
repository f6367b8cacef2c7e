"""Pins for the oracle's plain definitions of phi_l (O1-O4) -- CPU only.

Each check ties the oracle to something other than itself: mpmath quadrature of the
integral definition (Eq. (3)), closed forms, brute-force index loops for the Kronecker
ordering (Eq. (6)), the Kronecker exponential identity (Eq. (7)), the recurrence
(Eq. (4)), the modified squaring identity (Eq. (29)) and cross-agreement of the four
independent evaluations.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import workloads as W
from oracle import phi as P


# ----------------------------------------------------------------------------- scalar

@pytest.mark.parametrize("l", [0, 1, 2, 3, 5, 8])
@pytest.mark.parametrize("z", [-40.0, -7.5, -3.9, -1.0, -0.3, 0.0, 0.2, 1.0, 2.5, 9.0])
def test_phi_scalar_vs_quadrature_of_definition(l, z):
    import mpmath as mp
    with mp.workdps(40):
        if l == 0:
            ref = mp.e ** z
        else:
            ref = mp.quad(lambda t: mp.e ** ((1 - t) * z) * t ** (l - 1) / mp.factorial(l - 1), [0, 1])
    got = float(P.phi_scalar(l, np.array([z]))[0])
    assert abs(got - float(ref)) <= 2e-15 * max(abs(float(ref)), 1e-300) + 1e-300


def test_phi_scalar_closed_forms():
    z = np.array([-30.0, -2.0, -0.5, 0.7, 3.0])
    assert np.allclose(P.phi_scalar(1, z), np.expm1(z) / z, rtol=1e-14, atol=0)
    assert np.allclose(P.phi_scalar(2, z), (np.expm1(z) - z) / z ** 2, rtol=1e-12, atol=0)
    assert P.phi_scalar(4, np.array([0.0]))[0] == pytest.approx(1 / 24, rel=1e-15)


# ----------------------------------------------------------------------------- Kronecker ordering

def test_kron_sum_matches_index_definition():
    rng = np.random.default_rng(1)
    ax, ay, az = rng.standard_normal((2, 2)), rng.standard_normal((3, 3)), rng.standard_normal((4, 4))
    v = rng.standard_normal(2 * 3 * 4)
    V = v.reshape(2, 3, 4)
    ref = np.zeros_like(V)
    for i in range(2):
        for j in range(3):
            for k in range(4):
                s = 0.0
                for q in range(2):
                    s += ax[i, q] * V[q, j, k]
                for q in range(3):
                    s += ay[j, q] * V[i, q, k]
                for q in range(4):
                    s += az[k, q] * V[i, j, q]
                ref[i, j, k] = s
    A = P.kron_sum_dense([ax, ay, az])
    assert np.allclose(A @ v, ref.ravel(), atol=1e-13)
    As = P.kron_sum_sparse([ax, ay, az])
    assert np.allclose(As @ v, ref.ravel(), atol=1e-13)


def test_exp_of_kron_sum_is_kron_of_exps():
    rng = np.random.default_rng(2)
    a, b = rng.standard_normal((3, 3)), rng.standard_normal((5, 5))
    lhs = scipy.linalg.expm(P.kron_sum_dense([a, b]))
    rhs = np.kron(scipy.linalg.expm(a), scipy.linalg.expm(b))
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12)
    v = rng.standard_normal(15)
    assert np.allclose(P.apply_kron([scipy.linalg.expm(a), scipy.linalg.expm(b)], v.reshape(3, 5)).ravel(),
                       rhs @ v, atol=1e-12)


# ----------------------------------------------------------------------------- O1 closed forms

def test_O1_diagonal_factors_match_scalar_phi():
    lx, ly = np.array([0.5, 3.0, 11.0]), np.array([0.1, 2.0, 7.0, 20.0])
    tau, p = 0.3, 4
    v = W.uniform_vector((3, 4), 5)
    out = P.phi_dense([np.diag(lx), np.diag(ly)], tau, v, p)
    z = -tau * (lx[:, None] + ly[None, :])
    for l in range(p + 1):
        ref = P.phi_scalar(l, z).ravel() * v
        assert np.allclose(out[l], ref, rtol=1e-13, atol=1e-15)


def test_O1_phi1_closed_form_matrix():
    """phi_1(M) v = M^{-1}(e^M - I) v for invertible M."""
    A = W.convdiff_factor(5)
    M = -0.05 * P.kron_sum_dense([A, A])
    v = W.uniform_vector((5, 5), 3)
    out = P.phi_dense_matrix(M, v, 2)
    ref1 = np.linalg.solve(M, scipy.linalg.expm(M) @ v - v)
    ref2 = np.linalg.solve(M, ref1 - v)
    assert np.allclose(out[1], ref1, rtol=1e-12, atol=1e-14)
    assert np.allclose(out[2], ref2, rtol=1e-11, atol=1e-14)


def test_O1_recurrence_eq4():
    fac = [W.convdiff_factor(6), W.laplacian_factor(5), W.convdiff_factor(4)]
    tau, p = 0.02, 5
    v = W.uniform_vector((6, 5, 4), 7)
    out = P.phi_dense(fac, tau, v, p)
    M = -tau * P.kron_sum_dense(fac)
    for l in range(p):
        lhs = out[l]
        rhs = M @ out[l + 1] + v / math.factorial(l)
        assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(lhs)


def test_O1_modified_squaring_identity_eq29():
    fac = [W.convdiff_factor(7), W.convdiff_factor(6)]
    tau, p = 0.01, 4
    v = W.uniform_vector((7, 6), 9)
    half = P.phi_dense(fac, tau / 2, v, p)
    full = P.phi_dense(fac, tau, v, p)
    Mh = -tau / 2 * P.kron_sum_dense(fac)
    eM = scipy.linalg.expm(Mh)
    for q in range(1, p + 1):
        rhs = eM @ half[q] + sum(half[j] / math.factorial(q - j) for j in range(1, q + 1))
        rhs /= 2.0 ** q
        assert np.linalg.norm(full[q] - rhs) <= 1e-12 * np.linalg.norm(full[q])


# ----------------------------------------------------------------------------- cross-agreement

@pytest.mark.parametrize("shape", [(3, 4), (2, 3, 2)])
def test_O1_matches_O4_mpmath(shape):
    rng = np.random.default_rng(11)
    fac = [rng.standard_normal((n, n)) + 2 * np.eye(n) for n in shape]
    v = W.uniform_vector(shape, 12)
    tau, p = 0.4, 3
    o1 = P.phi_dense(fac, tau, v, p)
    o4 = P.phi_mpmath(fac, tau, v, p)
    for l in range(p + 1):
        assert P.rel_err_2(o1[l], o4[l]) <= 1e-13


def test_O3_matches_O1_nonsymmetric_3d():
    fac = [W.convdiff_factor(n) for n in (6, 5, 4)]
    tau, p = 1e-2, 3
    v = W.uniform_vector((6, 5, 4), 0)
    o1 = P.phi_dense(fac, tau, v, p)
    o3 = P.phi_sparse(fac, tau, v, p)
    for l in range(p + 1):
        assert P.rel_err_2(o3[l], o1[l]) <= 1e-13
    sub = P.phi_sparse(fac, tau, v, p, orders=[3, 0])
    assert P.rel_err_2(sub[0], o1[3]) <= 1e-13 and P.rel_err_2(sub[1], o1[0]) <= 1e-13


def test_O2_dirichlet_matches_O1():
    shape, coeffs = (5, 6, 7), (1.0, 0.5, 0.25)
    fac = [W.laplacian_factor(n, c) for n, c in zip(shape, coeffs)]
    tau, p = 2e-3, 3
    v = W.uniform_vector(shape, 4)
    o1 = P.phi_dense(fac, tau, v, p)
    o2 = P.phi_spectral_dirichlet(shape, coeffs, tau, v, p)
    for l in range(p + 1):
        assert P.rel_err_2(o2[l], o1[l]) <= 1e-13


def test_O2_periodic_matches_O1():
    shape = (8, 6)
    fac = [W.periodic_diffusion_factor(n, 0.3) for n in shape]
    tau, p = 1e-2, 2
    v = W.uniform_vector(shape, 6)
    o1 = P.phi_dense(fac, tau, v, p)
    o2 = P.phi_spectral_periodic(shape, (0.3, 0.3), tau, v, p)
    for l in range(p + 1):
        assert P.rel_err_2(o2[l], o1[l]) <= 1e-13


def test_O1_phi0_is_kron_of_1d_exponentials():
    fac = [W.convdiff_factor(n) for n in (4, 3, 5)]
    tau = 0.05
    v = W.uniform_vector((4, 3, 5), 8)
    o1 = P.phi_dense(fac, tau, v, 1)
    ref = P.apply_kron([scipy.linalg.expm(-tau * a) for a in fac], v.reshape(4, 3, 5)).ravel()
    assert P.rel_err_2(o1[0], ref) <= 1e-13
