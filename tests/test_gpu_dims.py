"""Kronecker sums of d != 2, 3 factors (Sec. 2 Remark: the mode-product form of Eq. (8) holds
in any dimension): one factor, and four to six factors, on the float64 and mixed paths,
against the dense augmented-matrix oracle (tiny sizes) and the DST-diagonalised oracle."""
import numpy as np
import pytest

import workloads as W
from oracle import erk as E
from oracle import phi as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _pk():
    import paper_2211_00696_gb300 as pk
    return pk


def _apply(fac, tau, p, tol, v, **kw):
    plan = _pk().Plan(fac, tau, p, tol, **kw)
    out = plan.apply(torch.from_numpy(v).cuda()).cpu().numpy()
    plan.check_status()
    info = plan.info()
    plan.close()
    return out, info


@pytest.mark.parametrize("shape", [(7,), (3, 4, 2, 5), (2, 3, 2, 2, 3), (2, 2, 2, 2, 2, 3)])
def test_small_any_dims_fp64_vs_dense_oracle(shape):
    rng = np.random.default_rng(len(shape))
    fac = [W.convdiff_factor(n) if i % 2 == 0 else W.laplacian_factor(n, 0.4) for i, n in enumerate(shape)]
    tau, p = 3e-3, 3
    v = rng.uniform(-1, 1, int(np.prod(shape)))
    exact = P.phi_dense(fac, tau, v, p)
    out, info = _apply(fac, tau, p, 1e-12, v)
    assert info["dims"] == len(shape) and info["n"][:len(shape)] == list(shape)
    for l in range(p + 1):
        assert P.rel_err_2(out[l], exact[l]) <= 1e-10, l


@pytest.mark.parametrize("shape,prec,tol,gate", [((16, 16, 16, 16), "fp64", 1e-12, 1e-10),
                                                  ((16, 32, 16, 16), "mixed", 1e-10, 1e-9),
                                                  ((16, 16, 16, 16, 16), "mixed", 1e-6, 1e-6),
                                                  ((48,), "mixed", 1e-10, 1e-9)])
def test_dims_vs_spectral_oracle(shape, prec, tol, gate):
    coeffs = [0.02 * (1 + 0.3 * d) for d in range(len(shape))]
    fac = [W.laplacian_factor(n, c) for n, c in zip(shape, coeffs)]
    tau, p = 1e-2, 2
    v = W.uniform_vector(shape, 21)
    exact = P.phi_spectral_dirichlet(shape, coeffs, tau, v, p)
    pk = _pk()
    out, info = _apply(fac, tau, p, tol, v, precision=pk.PREC_FP64 if prec == "fp64" else pk.PREC_OZAKI_BF16)
    for l in range(p + 1):
        assert P.rel_err_2(out[l], exact[l]) <= gate, (l, info)


def test_integrator_in_four_dimensions():
    shape, coeff, tau, nsteps = (16, 16, 16, 16), 0.01, 1e-2, 3
    fac = [W.laplacian_factor(n, coeff) for n in shape]
    u0 = W.uniform_vector(shape, 22, -0.7, 0.7)
    phi = lambda t, v, p: P.phi_spectral_dirichlet(shape, [coeff] * 4, t, v, p)
    ref = E.integrate(E.rk2(), u0, tau, nsteps, E.allen_cahn, lambda v: E.kron_sum_apply(fac, v), phi)
    pk = _pk()
    it = pk.Integrator(fac, tau, pk.ERK_RK2, 1e-12)
    U = torch.from_numpy(u0.copy()).cuda()
    it.step(U, nsteps)
    got = U.cpu().numpy()
    it.close()
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_seven_factors_rejected():
    pk = _pk()
    with pytest.raises(pk.PhikronError):
        pk.Plan([np.eye(2)] * 7, 1e-2, 1, 1e-8)
