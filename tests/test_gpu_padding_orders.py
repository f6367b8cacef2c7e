"""The mixed (tensor-core) path on sizes that are not multiples of 16 and on high phi orders.

Padding: a factor of size n is padded to the next multiple of 16 as diag(A^d, 0); its
exponentials are diag(e^{cA^d}, I), so a zero-padded input stays zero on the pad and the
leading block of every result is phi_l(-tau A) v.  Checked on the paper's 2^r - 1 grids (Sec. 4,
Tables 2 and 4: 15, 31, 63, 127 points per dimension) against the spectral oracle (O2), on
ragged nonsymmetric shapes (sizes below 16 included) against the sparse augmented-matrix oracle
(O3) and against the float64 GPU path with the same (s, m), with skip_phi0 and half-step outputs.

Orders: l_max up to 20 (the paper's range, Sec. 4) against the float64 path with the same
(s, m) and against the dense oracle (O1).  Gates as in test_gpu_mixed.py: 5 slices 5e-10 against
the float64 path; the plan tolerance plus the digit error against the definition.
"""
import numpy as np
import pytest

import workloads as W
from oracle import phi as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

BOUND = {3: 5e-6, 4: 5e-8, 5: 5e-10, 6: 5e-12}


def _pk():
    import paper_2211_00696_gb300 as pk
    return pk


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


@pytest.mark.parametrize("n,slices,tol,gate", [(15, 5, 1e-10, 1e-9), (31, 5, 1e-10, 1e-9), (63, 4, 1e-9, 1e-8),
                                               (127, 4, 1e-9, 1e-8)])
def test_paper_grids_laplace3d_vs_spectral(n, slices, tol, gate):
    pk = _pk()
    coeff, tau, p = 1.0, 1e-4 * (32.0 / (n + 1)) ** 2, 3
    shape = (n, n, n)
    fac = [W.laplacian_factor(n, coeff)] * 3
    v = W.uniform_vector(shape, 61)
    plan = pk.Plan(fac, tau, p, tol, precision=pk.PREC_OZAKI_BF16, slices=slices)
    out = plan.apply(_dev(v.ravel())).cpu().numpy()
    plan.check_status()
    exact = P.phi_spectral_dirichlet(shape, [coeff] * 3, tau, v, p)
    errs = [P.rel_err_2(out[l], exact[l].ravel()) for l in range(p + 1)]
    print(f"n={n}: (s,m)=({plan.info()['s']},{plan.info()['m']}) errors {errs}")
    assert max(errs) <= gate
    plan.close()


@pytest.mark.parametrize("shape", [(17, 33, 9), (40, 24), (5, 50, 20), (100,), (12, 10, 8, 6)])
def test_ragged_nonsymmetric_vs_oracle_and_float64(shape):
    pk = _pk()
    fac = [W.convdiff_factor(n) for n in shape]
    v = W.uniform_vector(shape, 62)
    tau, p = 1e-2, 3
    plan = pk.Plan(fac, tau, p, 1e-10, precision=pk.PREC_OZAKI_BF16, slices=5)
    info = plan.info()
    out = plan.apply(_dev(v.ravel())).cpu().numpy()
    plan.check_status()
    ref = pk.Plan(fac, tau, p, 1e-10, force_s=info["s"], force_m=info["m"])
    r64 = ref.apply(_dev(v.ravel())).cpu().numpy()
    exact = P.phi_sparse(fac, tau, v, p)
    for l in range(p + 1):
        assert P.rel_err_2(out[l], r64[l]) <= BOUND[5], (shape, l)
        assert P.rel_err_2(out[l], exact[l].ravel()) <= 1e-9, (shape, l)
    plan.close()
    ref.close()


def test_padding_with_skip_phi0_and_half_step():
    pk = _pk()
    shape = (20, 36, 44)
    fac = [W.laplacian_factor(n, 0.5) for n in shape]
    v = W.uniform_vector(shape, 63)
    tau, p = 2e-4, 2
    # skip_phi0: the phi_0 slot is left untouched
    plan = pk.Plan(fac, tau, p, 1e-10, precision=pk.PREC_OZAKI_BF16, slices=5, skip_phi0=True)
    out = torch.full((p + 1, v.size), 7.0, dtype=torch.float64, device="cuda")
    plan.apply(_dev(v.ravel()), out)
    out = out.cpu().numpy()
    plan.check_status()
    exact = P.phi_spectral_dirichlet(shape, [0.5] * 3, tau, v, p)
    assert np.all(out[0] == 7.0)
    for l in range(1, p + 1):
        assert P.rel_err_2(out[l], exact[l].ravel()) <= 1e-9
    plan.close()
    # half-step outputs phi_l(-tau/2 A) v after the phi_l(-tau A) v
    plan = pk.Plan(fac, tau, p, 1e-10, precision=pk.PREC_OZAKI_BF16, slices=5, half_step=True)
    out = plan.apply(_dev(v.ravel())).cpu().numpy()
    plan.check_status()
    half = P.phi_spectral_dirichlet(shape, [0.5] * 3, tau / 2, v, p)
    for l in range(p + 1):
        assert P.rel_err_2(out[l], exact[l].ravel()) <= 1e-9
        assert P.rel_err_2(out[p + 1 + l], half[l].ravel()) <= 1e-9
    plan.close()


@pytest.mark.parametrize("p", [9, 12, 20])
def test_high_orders_vs_float64_and_dense(p):
    """l_max up to 20: weighted sums and the squaring recurrence with up to 20 orders."""
    pk = _pk()
    shape = (16, 32)
    fac = [W.convdiff_factor(16), W.laplacian_factor(32, 0.3)]
    v = W.uniform_vector(shape, 64)
    tau = 2e-2
    # Algorithm 5 prefers s = 0 for p this large (each squaring step costs p actions); two
    # forced squaring steps make the recurrence of Eq. (29) run over all p orders
    plan = pk.Plan(fac, tau, p, 1e-10, precision=pk.PREC_OZAKI_BF16, slices=5, force_s=2, force_m=16)
    info = plan.info()
    assert (info["s"], info["m"]) == (2, 16)
    out = plan.apply(_dev(v.ravel())).cpu().numpy()
    plan.check_status()
    ref = pk.Plan(fac, tau, p, 1e-10, force_s=info["s"], force_m=info["m"])
    r64 = ref.apply(_dev(v.ravel())).cpu().numpy()
    exact = P.phi_dense(fac, tau, v.ravel(), p)
    for l in range(p + 1):
        assert P.rel_err_2(out[l], r64[l]) <= BOUND[5], l
        assert P.rel_err_2(out[l], exact[l]) <= 1e-9, l
    plan.close()
    ref.close()


def test_fused_weights_on_a_padded_plan_is_bitwise_the_separate_passes(monkeypatch):
    pk = _pk()
    shape = (24, 40, 100)      # padded to 32 x 48 x 112: the fused last pass over 112 rows
    fac = [W.convdiff_factor(n) for n in shape]
    v = W.uniform_vector(shape, 65)
    monkeypatch.setenv("PHIKRON_FUSED_WEIGHTS", "1")
    a_plan = pk.Plan(fac, 1e-2, 3, 1e-9, precision=pk.PREC_OZAKI_BF16, slices=4)
    monkeypatch.setenv("PHIKRON_FUSED_WEIGHTS", "0")
    b_plan = pk.Plan(fac, 1e-2, 3, 1e-9, precision=pk.PREC_OZAKI_BF16, slices=4)
    assert a_plan.info()["fused_weights"] == 1 and b_plan.info()["fused_weights"] == 0
    a = a_plan.apply(_dev(v.ravel())).cpu().numpy()
    b = b_plan.apply(_dev(v.ravel())).cpu().numpy()
    assert np.array_equal(a, b)
    a_plan.close()
    b_plan.close()
