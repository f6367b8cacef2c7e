"""Pins for the oracle's measured criterion, (s, m) search and selector network (CPU), and
parity of the library's host-side criterion/search with the oracle."""
import numpy as np
import pytest
import scipy.linalg

import workloads as W
from oracle import phi as P
from oracle import planner as PL
from oracle import quadrature as Q
from oracle import selector as OS


def _method_matrix_error(fac, tau, p, s, m):
    """||Phi_j(M) - phi_j(M)||_2 (largest over j) for the method with (s, m), via the oracle's
    restated Algorithm 6 applied to every unit vector."""
    N = int(np.prod([a.shape[0] for a in fac]))
    worst = 0.0
    exact_cols, got_cols = [], []
    for i in range(N):
        e = np.zeros(N)
        e[i] = 1.0
        got_cols.append(Q.alg6_phiquadmv(fac, tau, e, p, 1e-12, s=s, m=m))
        exact_cols.append(P.phi_dense(fac, tau, e, p))
    for j in range(1, p + 1):
        G = np.array([g[j] for g in got_cols]).T
        X = np.array([x[j] for x in exact_cols]).T
        worst = max(worst, np.linalg.norm(G - X, 2))
    return worst


@pytest.mark.parametrize("s,m", [(0, 3), (1, 4), (2, 3), (0, 6)])
def test_criterion_bounds_matrix_error_for_symmetric_operator(s, m):
    fac = [W.laplacian_factor(n, c) for n, c in ((4, 1.0), (3, 0.5), (5, 0.3))]
    tau, p = 0.02, 3
    M = -tau * P.kron_sum_dense(fac)
    lam = np.linalg.eigvalsh(M)
    actual = _method_matrix_error(fac, tau, p, s, m)
    crit = OS.criterion(lam.min(), lam.max(), p, s, m, npts=2000)
    assert actual <= crit * (1 + 1e-6) + 1e-15
    # and it is attained (the scalar error at the eigenvalues is the matrix error)
    assert crit <= 3.0 * actual + 1e-14


def test_search_returns_minimal_nodes_for_its_scaling():
    rng = np.random.default_rng(3)
    for _ in range(8):
        zlo = -10 ** rng.uniform(-1, 3.5)
        p = int(rng.integers(1, 5))
        tol = float(rng.choice([1e-6, 1e-8, 1e-10]))
        s, m, cost = OS.search(zlo, 0.0, p, tol)
        assert cost == m + s * p
        assert OS.criterion(zlo, 0.0, p, s, m) <= tol
        if m > 2:
            assert OS.criterion(zlo, 0.0, p, s, m - 1) > tol


def test_network_gradient_matches_finite_differences():
    rng = np.random.default_rng(8)
    params = rng.standard_normal(OS.n_params()) * 0.2
    X = rng.standard_normal((16, 8))
    ys = rng.integers(0, 21, 16)
    ym = rng.integers(2, 33, 16)
    g = OS.grads(params, X, ys, ym)
    idx = rng.choice(len(params), 40, replace=False)
    for i in idx:
        h = 1e-6
        pp, pm = params.copy(), params.copy()
        pp[i] += h
        pm[i] -= h
        fd = (OS.loss(pp, X, ys, ym) - OS.loss(pm, X, ys, ym)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), i


def test_library_criterion_and_search_match_oracle():
    import ctypes as C
    import paper_2211_00696_gb300 as pk
    from paper_2211_00696_gb300 import phikron as B
    L = pk.lib()
    err = C.c_double()
    for zlo, p, s, m in [(-30.0, 3, 2, 8), (-1500.0, 3, 6, 7), (-0.5, 1, 0, 3), (-2e4, 4, 9, 12)]:
        assert L.phikron_selector_criterion(zlo, 0.0, p, s, m, 128, C.byref(err)) == 0
        ref = OS.criterion(zlo, 0.0, p, s, m)
        assert abs(err.value - ref) <= 1e-8 * ref + 1e-15   # scalar roundoff ~1e-16 absolute
    rng = np.random.default_rng(5)
    n = 40
    zlo = -10 ** rng.uniform(-2, 4.5, n)
    zhi = np.zeros(n)
    p = rng.integers(1, 5, n).astype(np.int32)
    tol = rng.choice([1e-6, 1e-8, 1e-10], n)
    so, mo, co = (np.zeros(n, np.int32) for _ in range(3))
    rc = L.phikron_selector_search(n, zlo.ctypes.data_as(B._DP), zhi.ctypes.data_as(B._DP), p.ctypes.data_as(B._IP),
                                   tol.ctypes.data_as(B._DP), 128, 4, so.ctypes.data_as(B._IP),
                                   mo.ctypes.data_as(B._IP), co.ctypes.data_as(B._IP))
    assert rc == 0
    for i in range(n):
        assert OS.search(zlo[i], zhi[i], int(p[i]), tol[i]) == (so[i], mo[i], co[i]), i


def test_measured_labels_never_cost_more_than_a_priori_plan_on_laplacians():
    """The measured criterion is tighter than Theorem 3.2's bound, so for these symmetric
    operators its cost-minimising (s, m) costs at most what Algorithm 5 plans (over a sample)."""
    from paper_2211_00696_gb300 import selector as S
    n, c, tau, p, tol = S.sample_problems(60, 11)
    s, m, cost = S.labels(n, c, tau, p, tol)
    worse = 0
    for i in range(60):
        alpha = tau[i] * np.sum(4.0 * c[i] * (n[i] + 1.0) ** 2)
        ps, pm, pc = PL.setup_quadrature(tol[i], int(p[i]), alpha)
        worse += cost[i] > pc
    assert worse == 0
