"""GPU parity of the mixed-precision path (split-BF16 tensor-core mode products,
float-float state) against the oracle.

Error model: each mode product is exact up to the digit truncation of its two operands,
about 2^(1 - 8*slices) relative to ||E||_inf max|x| per product, and the float-float state
carries ~2^-48.  With ~(m + s*p + 1)*dims products per apply the bounds used here are
slices 3: 5e-6, 4: 5e-8, 5: 5e-10, 6: 5e-12 relative 2-norm error per phi_l against the
float64 GPU path with the same (s, m), plus the quadrature tolerance against the exact
definition.
"""
import numpy as np
import pytest

import workloads as W
from oracle import phi as P
from oracle import quadrature as Q

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

BOUND = {3: 5e-6, 4: 5e-8, 5: 5e-10, 6: 5e-12}


def _pk():
    import paper_2211_00696_gb300 as pk
    return pk


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _mixed_and_fp64(factors, tau, l_max, tol, v, slices, **kw):
    pk = _pk()
    pm = pk.Plan(factors, tau, l_max, tol, precision=pk.PREC_OZAKI_BF16, slices=slices, **kw)
    info = pm.info()
    pf = pk.Plan(factors, tau, l_max, tol, force_s=info["s"], force_m=info["m"], **kw)
    om = pm.apply(_dev(v)).cpu().numpy()
    of = pf.apply(_dev(v)).cpu().numpy()
    pm.check_status()
    return om, of, info


@pytest.mark.parametrize("slices", [3, 4, 5, 6])
def test_convdiff3d_mixed_vs_fp64_path(slices):
    shape = (32, 48, 64)
    fac = [W.convdiff_factor(n) for n in shape]
    v = W.uniform_vector(shape, 0)
    om, of, info = _mixed_and_fp64(fac, 1e-2, 3, 1e-10, v, slices)
    assert info["slices"] == slices
    for l in range(4):
        assert P.rel_err_2(om[l], of[l]) <= BOUND[slices], (slices, l, P.rel_err_2(om[l], of[l]))


@pytest.mark.parametrize("kernel", ["ws", "db", "classic"])
@pytest.mark.parametrize("slices", [3, 4, 5])
def test_mode_kernel_variants_vs_fp64_path(kernel, slices, monkeypatch):
    """Every mode-kernel variant (warp-specialised default, double-buffered, single-role) at
    2- and 3-stage operand rings (up to 4 slices: three stages) and several tiles per CTA:
    n >= 64 on every axis so that the double-buffered kernel is eligible; 160 = 128 + 32 puts a
    second E row block and a ragged tail on one axis."""
    if kernel != "ws":
        monkeypatch.setenv("PHIKRON_MODE_KERNEL", kernel)
    shape = (64, 160, 96)
    fac = [W.convdiff_factor(n) for n in shape]
    v = W.uniform_vector(shape, 9)
    om, of, info = _mixed_and_fp64(fac, 1e-2, 3, 1e-10, v, slices)
    for l in range(4):
        assert P.rel_err_2(om[l], of[l]) <= BOUND[slices], (kernel, slices, l, P.rel_err_2(om[l], of[l]))


def test_convdiff3d_mixed_vs_exact_definition():
    shape = (16, 32, 48)
    fac = [W.convdiff_factor(n) for n in shape]
    v = W.uniform_vector(shape, 1)
    exact = P.phi_sparse(fac, 1e-2, v, 3)
    pk = _pk()
    plan = pk.Plan(fac, 1e-2, 3, 1e-10, precision=pk.PREC_OZAKI_BF16)
    out = plan.apply(_dev(v)).cpu().numpy()
    plan.check_status()
    assert plan.info()["slices"] == 5
    for l in range(4):
        assert P.rel_err_2(out[l], exact[l]) <= 1e-9, l


def test_laplace2d_config1_mixed_vs_dense_oracle():
    prob = W.laplace2d()
    v = prob.vector()
    exact = P.phi_dense(prob.factors, prob.tau, v, prob.l_max)
    pk = _pk()
    plan = pk.Plan(prob.factors, prob.tau, prob.l_max, prob.tol, precision=pk.PREC_OZAKI_BF16)
    out = plan.apply(_dev(v)).cpu().numpy()
    plan.check_status()
    for l in range(prob.l_max + 1):
        assert P.rel_err_2(out[l], exact[l]) <= 1e-9, l


@pytest.mark.parametrize("shape", [(48, 80, 16), (112, 16), (16, 16, 16), (128, 32, 96)])
def test_ragged_shapes_match_algorithm6(shape):
    fac = [W.convdiff_factor(n) for n in shape]
    v = W.uniform_vector(shape, 2)
    pk = _pk()
    plan = pk.Plan(fac, 5e-3, 3, 1e-10, precision=pk.PREC_OZAKI_BF16, slices=6)
    info = plan.info()
    out = plan.apply(_dev(v)).cpu().numpy()
    plan.check_status()
    ref = Q.alg6_phiquadmv(fac, 5e-3, v, 3, 1e-10, s=info["s"], m=info["m"])
    for l in range(4):
        assert P.rel_err_2(out[l], ref[l]) <= 1e-11, (shape, l)


def test_mixed_edge_cases():
    pk = _pk()
    fac = [W.convdiff_factor(32), W.laplacian_factor(48)]
    v = W.uniform_vector((32, 48), 3)
    # phi_0 only
    plan = pk.Plan(fac, 1e-2, 0, 1e-10, precision=pk.PREC_OZAKI_BF16, slices=6)
    out = plan.apply(_dev(v)).cpu().numpy()
    assert P.rel_err_2(out[0], P.phi_dense(fac, 1e-2, v, 0)[0]) <= 1e-11
    # s = 0 (weighted sums write float64 directly)
    plan = pk.Plan(fac, 1e-2, 2, 1e-10, precision=pk.PREC_OZAKI_BF16, slices=6, force_s=0, force_m=24)
    out = plan.apply(_dev(v)).cpu().numpy()
    exact = P.phi_dense(fac, 1e-2, v, 2)
    for l in range(3):
        assert P.rel_err_2(out[l], exact[l]) <= 1e-10
    # tau = 0: phi_l(0) v = v / l!  (digits are relative to the vector's max: 2-norm error)
    plan = pk.Plan(fac, 0.0, 3, 1e-10, precision=pk.PREC_OZAKI_BF16, slices=6)
    out = plan.apply(_dev(v)).cpu().numpy()
    for l, f in enumerate([1, 1, 2, 6]):
        assert P.rel_err_2(out[l], v / f) <= 1e-13
    # zero input vector
    out = plan.apply(_dev(np.zeros_like(v))).cpu().numpy()
    assert not np.any(out)
    plan.check_status()


def test_mixed_rejects_unsupported_sizes():
    pk = _pk()
    # padded plans (a size not a multiple of 16) are not batched
    padded = pk.Plan([W.laplacian_factor(20), W.laplacian_factor(32)], 1e-3, 2, 1e-8, precision=pk.PREC_OZAKI_BF16)
    with pytest.raises(pk.PhikronError) as e:
        pk.Batch([padded], nrhs=1)
    assert e.value.code == pk.phikron.ENOTSUP
    padded.close()
    with pytest.raises(pk.PhikronError):     # above the 4096 limit of the mixed path
        pk.Plan([W.laplacian_factor(4112), W.laplacian_factor(16)], 1e-6, 1, 1e-8, precision=pk.PREC_OZAKI_BF16)


@pytest.mark.parametrize("n,prec,tol", [(512, "mixed", 1e-10), (2048, "mixed", 1e-6), (2048, "mixed", 1e-10),
                                        (2048, "fp64", 1e-10)])
def test_large_n_periodic_2d_vs_spectral(n, prec, tol):
    """Long contractions (K = n up to 2048, 64 K-chunks, 16 E row blocks) on the 2D periodic
    diffusion operator of the Allen-Cahn workload (eps^2 = 1e-4, tau = 1e-2, phi_0 and phi_1)
    against the DFT-diagonalised oracle; the gate is the plan tolerance."""
    import time
    pk = _pk()
    coeff, tau, p = 1e-4, 1e-2, 1
    fac = [W.periodic_diffusion_factor(n, coeff)] * 2
    v = W.uniform_vector((n, n), 7)
    exact = P.phi_spectral_periodic((n, n), [coeff] * 2, tau, v, p)
    t0 = time.perf_counter()
    plan = pk.Plan(fac, tau, p, tol, precision=pk.PREC_OZAKI_BF16 if prec == "mixed" else pk.PREC_FP64)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    out = plan.apply(_dev(v)).cpu().numpy()
    plan.check_status()
    errs = [P.rel_err_2(out[l], exact[l]) for l in range(p + 1)]
    print(f"n={n} {prec} tol={tol:g}: plan {plan_s:.2f} s, errors {errs}")
    assert max(errs) <= tol
    assert plan_s < 20.0
