"""Adaptive Clenshaw-Curtis (Algorithm 2 inside Algorithm 3) on the float64 path: the node
count the library settles on equals the oracle's (same nested rules, same stopping test), the
outputs match the oracle's restatement and the exact definition, the node cap reports
ENOTCONVERGED, and the 128^3 convection-diffusion workload meets its tolerance."""
import numpy as np
import pytest

import workloads as W
from oracle import phi as P
from oracle import quadrature as Q

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _pk():
    import paper_2211_00696_gb300 as pk
    return pk


@pytest.mark.parametrize("tol", [1e-6, 1e-10, 1e-13])
def test_adaptive_matches_oracle_restatement(tol):
    pk = _pk()
    fac = [W.convdiff_factor(12), W.laplacian_factor(10, 0.6), W.convdiff_factor(8)]
    tau, p = 1e-2, 3
    v = W.uniform_vector((12, 10, 8), 31)
    plan = pk.Plan(fac, tau, p, tol, quad=pk.QUAD_CC_ADAPTIVE)
    info = plan.info()
    out = plan.apply(torch.from_numpy(v).cuda()).cpu().numpy()
    after = plan.info()
    ref, st = Q.alg6_phiquadmv(fac, tau, v, p, tol, s=info["s"], m=1, rule="cc_adaptive", return_stages=True)
    # stopping decisions agree unless the estimate sits within 1% of tol
    if abs(st["err"] - tol) > 0.01 * tol:
        assert after["adaptive_nodes"] == st["nodes"], (after["adaptive_nodes"], st)
    exact = P.phi_dense(fac, tau, v, p)
    for l in range(p + 1):
        assert P.rel_err_2(out[l], ref[l]) <= 1e-12 + 1e-3 * tol, l
        assert P.rel_err_2(out[l], exact[l]) <= 10 * tol + 1e-13, l
    assert after["adaptive_err"] <= tol
    plan.close()


def test_adaptive_node_cap_reports_not_converged():
    pk = _pk()
    fac = [W.laplacian_factor(16, 1.0)] * 2
    v = W.uniform_vector((16, 16), 32)
    plan = pk.Plan(fac, 2e-2, 2, 1e-14, quad=pk.QUAD_CC_ADAPTIVE, force_s=0, force_m=13)
    with pytest.raises(pk.PhikronError) as e:
        plan.apply(torch.from_numpy(v).cuda())
    assert e.value.code == pk.phikron.ENOTCONVERGED
    assert plan.info()["adaptive_nodes"] == 13
    plan.close()


def test_adaptive_rejects_mixed_path():
    pk = _pk()
    with pytest.raises(pk.PhikronError):
        pk.Plan([W.laplacian_factor(16)] * 2, 1e-3, 2, 1e-8, quad=pk.QUAD_CC_ADAPTIVE,
                precision=pk.PREC_OZAKI_BF16)


def test_adaptive_convdiff3d_128_against_stored_oracle_samples():
    """The 128^3 convection-diffusion workload against the stored O3 samples (sampled relative
    error normalised like the full 2-norm: rms(diff) / rms(phi_l)), gated at 1e-10, the
    float64 path's accuracy target on this workload."""
    import os
    import sys
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
    from make_convdiff_samples import load
    pk = _pk()
    prob = W.convdiff3d()
    idx, vals, norm2, _ = load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                            "convdiff3d_n128_tau1e-2_seed0_samples.txt"))
    plan = pk.Plan(prob.factors, prob.tau, prob.l_max, 1e-10, quad=pk.QUAD_CC_ADAPTIVE)
    out = plan.apply(torch.from_numpy(prob.vector()).cuda()).cpu().numpy()
    info = plan.info()
    for l in range(prob.l_max + 1):
        d = out[l][idx] - vals[l]
        err = np.sqrt(np.mean(d * d)) / (norm2[l] / np.sqrt(prob.N))
        print(f"phi_{l}: sampled relative error {err:.3e}")
        assert err <= 1e-10, (l, err, info["adaptive_nodes"])
    print(f"adaptive CC 128^3: s={info['s']} nodes={info['adaptive_nodes']} err={info['adaptive_err']:.2e}")
    plan.close()
