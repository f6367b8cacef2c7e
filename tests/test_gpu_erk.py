"""GPU parity of the exponential Runge-Kutta drivers (Eq. (RK), Table RK) through the C ABI
against the oracle's tableau steps (oracle/erk.py, phi-actions from the spectral oracles),
the exact propagation of the linear problem, the observed orders on the GPU, and the
Allen-Cahn configuration (2048^2 periodic, eps = 0.01, tau = 1e-2) mixed vs float64.

Tolerances: a step adds tau*phi(...)D with |tau D| up to ~tau*||A||*|u|, so a relative
phi-action error e becomes ~e*tau*||A|| in u per step; the float64 plans use tol 1e-12 and the
mixed plans 1e-10, and the gates below allow that amplification over the steps taken."""
import numpy as np
import pytest

import workloads as W
from oracle import erk as E
from oracle import phi as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

METHODS = {"euler": 1, "rk2": 2, "rk3": 3}


def _pk():
    import paper_2211_00696_gb300 as pk
    return pk


def _run(fac, u0, tau, nsteps, method, prec, tol, nonlin=1):
    pk = _pk()
    it = pk.Integrator(fac, tau, METHODS[method], tol, nonlinearity=nonlin,
                       precision=pk.PREC_FP64 if prec == "fp64" else pk.PREC_OZAKI_BF16)
    U = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
    it.step(U, nsteps)
    torch.cuda.synchronize()
    it.check_status()
    info = it.info()
    it.close()
    return U.cpu().numpy(), info


@pytest.mark.parametrize("method", ["euler", "rk2", "rk3"])
@pytest.mark.parametrize("prec,tol,gate", [("fp64", 1e-12, 1e-10), ("mixed", 1e-10, 1e-8)])
def test_periodic_allen_cahn_matches_oracle(method, prec, tol, gate):
    n, eps, tau, nsteps = 64, 0.05, 1e-2, 6
    fac = [W.periodic_diffusion_factor(n, eps * eps)] * 2
    u0 = W.uniform_vector((n, n), 11, -0.5, 0.5)
    phi = lambda t, v, p: P.phi_spectral_periodic((n, n), [eps * eps] * 2, t, v, p)
    ref = E.integrate(E.TABLEAUS[method](), u0, tau, nsteps, E.allen_cahn,
                      lambda v: E.kron_sum_apply(fac, v), phi)
    got, info = _run(fac, u0, tau, nsteps, method, prec, tol)
    assert info["applies_per_step"] == {"euler": 1, "rk2": 2, "rk3": 5}[method]
    assert np.linalg.norm(got - ref) <= gate * np.linalg.norm(ref)


@pytest.mark.parametrize("method", ["euler", "rk3"])
def test_dirichlet_3d_allen_cahn_matches_oracle(method):
    shape, coeff, tau, nsteps = (16, 32, 16), 0.02, 5e-3, 4
    fac = [W.laplacian_factor(n, coeff) for n in shape]
    u0 = W.uniform_vector(shape, 12, -0.8, 0.8)
    phi = lambda t, v, p: P.phi_spectral_dirichlet(shape, [coeff] * 3, t, v, p)
    ref = E.integrate(E.TABLEAUS[method](), u0, tau, nsteps, E.allen_cahn,
                      lambda v: E.kron_sum_apply(fac, v), phi)
    for prec, tol, gate in (("fp64", 1e-12, 1e-10), ("mixed", 1e-10, 1e-8)):
        got, _ = _run(fac, u0, tau, nsteps, method, prec, tol)
        assert np.linalg.norm(got - ref) <= gate * np.linalg.norm(ref), prec


def test_linear_problem_is_propagated_exactly():
    """f = 0: every method gives e^{-k tau A} u after k steps (CSR apply of A and the stage
    combinations checked against the DFT oracle)."""
    n, coeff, tau, nsteps = 48, 2e-3, 2e-2, 5
    fac = [W.periodic_diffusion_factor(n, coeff)] * 2
    u0 = W.uniform_vector((n, n), 13)
    ref = P.phi_spectral_periodic((n, n), [coeff] * 2, nsteps * tau, u0, 0)[0]
    for method in METHODS:
        got, _ = _run(fac, u0, tau, nsteps, method, "fp64", 1e-12, nonlin=0)
        assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref), method


@pytest.mark.parametrize("method,order", [("euler", 1), ("rk2", 2), ("rk3", 3)])
def test_observed_order_on_gpu(method, order):
    """The oracle test's stiff Allen-Cahn problem (8 x 7 Dirichlet grid, smooth data, T = 1),
    integrated by the library; reference from the oracle's RK3 at 512 steps."""
    n1, n2 = 8, 7
    fac = [W.laplacian_factor(n1, 0.1), W.laplacian_factor(n2, 0.1)]
    x = np.arange(1, n1 + 1) / (n1 + 1)
    y = np.arange(1, n2 + 1) / (n2 + 1)
    u0 = (0.9 * np.outer(np.sin(np.pi * x), np.sin(np.pi * y))
          + 0.3 * np.outer(np.sin(2 * np.pi * x), np.sin(3 * np.pi * y))).ravel()
    T = 1.0
    ref = E.integrate(E.rk3(), u0, T / 512, 512, E.allen_cahn, lambda v: E.kron_sum_apply(fac, v),
                      lambda t, v, p: P.phi_dense(fac, t, v, p))
    errs = []
    for nsteps in (16, 32, 64):
        got, _ = _run(fac, u0, T / nsteps, nsteps, method, "fp64", 1e-13)
        errs.append(np.max(np.abs(got - ref)))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) >= order - 0.15 and max(rates) <= order + 0.3, (errs, rates)


@pytest.mark.parametrize("method", ["euler", "rk2"])
def test_allen_cahn_2048_mixed_vs_fp64(method):
    """The 2048^2 periodic Allen-Cahn configuration (eps = 0.01, tau = 1e-2, u0 ~ U(-0.05, 0.05)
    seed 4) for 20 steps: mixed vs float64 GPU final state <= 1e-6 relative, and the float64
    path against the oracle's tableau steps with DFT phi-actions."""
    nsteps, tau, eps = 20, 1e-2, 0.01
    a, u0 = W.allen_cahn2d()
    fac = [a, a]
    got64, _ = _run(fac, u0, tau, nsteps, method, "fp64", 1e-12)
    gotmx, _ = _run(fac, u0, tau, nsteps, method, "mixed", 1e-10)
    assert np.linalg.norm(gotmx - got64) <= 1e-6 * np.linalg.norm(got64)
    n = a.shape[0]
    phi = lambda t, v, p: P.phi_spectral_periodic((n, n), [eps * eps] * 2, t, v, p)
    ref = E.integrate(E.TABLEAUS[method](), u0, tau, nsteps, E.allen_cahn,
                      lambda v: E.kron_sum_apply(fac, v), phi)
    assert np.linalg.norm(got64 - ref) <= 1e-10 * np.linalg.norm(ref)
