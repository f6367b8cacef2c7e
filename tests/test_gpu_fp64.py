"""GPU parity of the float64 path against the oracle (element by element).

Tolerance: the spec gate for the float64 path is relative 2-norm error <= 1e-10 per
phi_l against the plain definition.  Against the oracle's restatement of Algorithm 6 with
the same (s, m) the two compute the same approximation, so they must agree to rounding:
<= 1e-12 relative (a few hundred float64 roundings through ~m+s*p Kronecker actions).
"""
import numpy as np
import pytest
import scipy.linalg

import workloads as W
from oracle import phi as P
from oracle import quadrature as Q

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _pk():
    import paper_2211_00696_gb300 as pk
    return pk


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


# ----------------------------------------------------------------------------- K1 expm

@pytest.mark.parametrize("n", [1, 5, 32, 70, 128])
def test_expm_batched_matches_scipy(n):
    pk = _pk()
    rng = np.random.default_rng(n)
    mats = [W.convdiff_factor(n), W.laplacian_factor(n), rng.standard_normal((n, n))]
    scales = [-0.01, -1e-3, 0.3, -2.5e-4, -0.08, 1.7]
    A = np.stack([mats[i % 3] for i in range(len(scales))])
    E = _pk().expm_batched(_dev(A), scales).cpu().numpy()
    for b, c in enumerate(scales):
        ref = scipy.linalg.expm(c * A[b])
        # degree-18 Taylor truncation < u at ||B||_1 <= 1; each of the s_b squarings can add a
        # few u (s_b = ceil(log2 ||cA||_1); scaling and squaring in numpy shows ~1.8e-13 at 9)
        sb = max(0, int(np.ceil(np.log2(abs(c) * np.abs(A[b]).sum(0).max()))))
        tol = 2e-14 * (5 + 5 * sb)
        assert np.linalg.norm(E[b] - ref) <= tol * max(1.0, np.linalg.norm(ref)), (b, c, sb)


def test_expm_batched_needs_squaring():
    rng = np.random.default_rng(7)
    A = rng.standard_normal((3, 48, 48))
    scales = [4.0, -9.0, 1.5]            # ||cA||_1 ~ 100-300: several squarings
    E = _pk().expm_batched(_dev(A), scales).cpu().numpy()
    for b, c in enumerate(scales):
        ref = scipy.linalg.expm(c * A[b])
        assert np.linalg.norm(E[b] - ref) <= 1e-11 * np.linalg.norm(ref)


# ----------------------------------------------------------------------------- K2 mode products

@pytest.mark.parametrize("shape", [(13, 70, 9), (64, 65, 3), (130, 1, 7), (40, 33)])
def test_kron_apply_f64_matches_oracle(shape):
    rng = np.random.default_rng(3)
    mats = [rng.standard_normal((n, n)) for n in shape]
    v = rng.standard_normal(int(np.prod(shape)))
    got = _pk().kron_apply_f64([_dev(m) for m in mats], _dev(v)).cpu().numpy()
    ref = P.apply_kron(mats, v.reshape(shape)).ravel()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


# ----------------------------------------------------------------------------- full path

def _run(factors, tau, l_max, tol, v, **kw):
    pk = _pk()
    plan = pk.Plan(factors, tau, l_max, tol, **kw)
    out = plan.apply(_dev(v)).cpu().numpy()
    return out, plan


def test_config1_laplace2d_fp64_vs_dense_oracle():
    prob = W.laplace2d()                      # n = 32, tau = 1e-3, phi_0..phi_3, tol 1e-10
    v = prob.vector()
    exact = P.phi_dense(prob.factors, prob.tau, v, prob.l_max)
    out, plan = _run(prob.factors, prob.tau, prob.l_max, prob.tol, v)
    info = plan.info()
    assert (info["s"], info["m"]) == (1, 9)
    for l in range(prob.l_max + 1):
        assert P.rel_err_2(out[l], exact[l]) <= 1e-10, l


def test_config1_matches_algorithm6_restated():
    prob = W.laplace2d()
    v = prob.vector()
    out, plan = _run(prob.factors, prob.tau, prob.l_max, prob.tol, v)
    info = plan.info()
    ref = Q.alg6_phiquadmv(prob.factors, prob.tau, v, prob.l_max, prob.tol, s=info["s"], m=info["m"])
    for l in range(prob.l_max + 1):
        assert P.rel_err_2(out[l], ref[l]) <= 1e-12


@pytest.mark.parametrize("shape,tau,l_max", [((10, 12, 9), 1e-2, 3), ((7, 66, 5), 3e-3, 4),
                                              ((17, 15), 5e-2, 2)])
def test_nonsymmetric_uneven_vs_dense_oracle(shape, tau, l_max):
    fac = [W.convdiff_factor(n) for n in shape]
    v = W.uniform_vector(shape, 5)
    exact = P.phi_dense(fac, tau, v, l_max)
    out, _ = _run(fac, tau, l_max, 1e-12, v)
    for l in range(l_max + 1):
        assert P.rel_err_2(out[l], exact[l]) <= 1e-10, l


def test_forced_scaling_and_nodes_match_algorithm6():
    shape = (9, 11, 8)
    fac = [W.convdiff_factor(n) for n in shape]
    v = W.uniform_vector(shape, 6)
    for s, m in [(0, 12), (3, 6), (6, 5)]:
        out, _ = _run(fac, 2e-2, 3, 1e-10, v, force_s=s, force_m=m)
        ref = Q.alg6_phiquadmv(fac, 2e-2, v, 3, 1e-10, s=s, m=m)
        for l in range(4):
            assert P.rel_err_2(out[l], ref[l]) <= 1e-12, (s, m, l)


def test_edge_cases_phi0_only_tau_zero_and_tiny_sizes():
    fac = [W.convdiff_factor(6), W.laplacian_factor(5)]
    v = W.uniform_vector((6, 5), 8)
    out, _ = _run(fac, 1e-2, 0, 1e-10, v)                  # phi_0 only
    assert P.rel_err_2(out[0], P.phi_dense(fac, 1e-2, v, 0)[0]) <= 1e-13
    out, plan = _run(fac, 0.0, 3, 1e-10, v)                # tau = 0: phi_l(0) = I/l!
    for l, f in enumerate([1, 1, 2, 6]):
        assert np.allclose(out[l], v / f, rtol=1e-14, atol=0)
    f1 = [np.array([[2.0]]), np.array([[0.5]]), np.array([[1.0]])]   # N = 1
    out, _ = _run(f1, 0.7, 3, 1e-12, np.array([0.3]))
    z = -0.7 * 3.5
    for l in range(4):
        assert out[l][0] == pytest.approx(0.3 * P.phi_scalar(l, np.array([z]))[0], rel=1e-11)


def test_apply_host_matches_device_apply():
    pk = _pk()
    prob = W.laplace2d(n=24)
    v = prob.vector()
    plan = pk.Plan(prob.factors, prob.tau, prob.l_max, prob.tol)
    dev = plan.apply(_dev(v)).cpu().numpy()
    host = plan.apply_host(v)
    assert np.array_equal(dev, host)


def test_apply_many_matches_single():
    pk = _pk()
    fac = [W.convdiff_factor(n) for n in (8, 9, 10)]
    plan = pk.Plan(fac, 1e-2, 3, 1e-10, max_rhs=3)
    V = np.stack([W.uniform_vector((8, 9, 10), s) for s in range(3)])
    many = plan.apply_many(_dev(V)).cpu().numpy()
    for r in range(3):
        one = plan.apply(_dev(V[r])).cpu().numpy()
        assert np.array_equal(many[r], one)
