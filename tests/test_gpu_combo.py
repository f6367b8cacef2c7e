"""sum_j phi_j(-tau A) b_j in one quadrature (the Remark after Algorithm 2) on the float64
path: against the oracle's restatement with the plan's own nodes and against the separate
phi-actions of the exact definition; plans with s > 0 and mixed plans are refused."""
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


@pytest.mark.parametrize("shape,p", [((12, 10, 8), 3), ((32, 48), 2), ((16, 16, 16), 4)])
def test_combo_matches_oracle_and_definition(shape, p):
    pk = _pk()
    fac = [W.convdiff_factor(n) if i == 0 else W.laplacian_factor(n, 0.3) for i, n in enumerate(shape)]
    tau = 1e-4
    N = int(np.prod(shape))
    B = np.stack([W.uniform_vector(shape, 40 + j) for j in range(p)])
    plan = pk.Plan(fac, tau, p, 1e-12)
    info = plan.info()
    assert info["s"] == 0
    x, w = plan.nodes()
    got = plan.apply_combo(torch.from_numpy(B).cuda()).cpu().numpy()
    ref = Q.remark_combo(fac, tau, list(B), x, w)
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    if N <= 2000:
        exact = sum(P.phi_dense(fac, tau, B[j - 1], p)[j] for j in range(1, p + 1))
        assert np.linalg.norm(got - exact) <= 1e-11 * np.linalg.norm(exact)
    # and the same sum from the ordinary apply, order by order
    outs = [plan.apply(torch.from_numpy(B[j - 1]).cuda()).cpu().numpy()[j] for j in range(1, p + 1)]
    assert np.linalg.norm(got - sum(outs)) <= 1e-12 * np.linalg.norm(got)
    plan.close()


def test_combo_refuses_scaled_and_mixed_plans():
    pk = _pk()
    fac = [W.laplacian_factor(16, 1.0)] * 2
    B = torch.zeros((2, 256), dtype=torch.float64, device="cuda")
    plan = pk.Plan(fac, 1.0, 2, 1e-10)
    assert plan.info()["s"] > 0
    with pytest.raises(pk.PhikronError) as e:
        plan.apply_combo(B)
    assert e.value.code == pk.phikron.EINVAL
    plan.close()
    plan = pk.Plan(fac, 1e-5, 2, 1e-8, precision=pk.PREC_OZAKI_BF16)
    with pytest.raises(pk.PhikronError) as e:
        plan.apply_combo(B)
    assert e.value.code == pk.phikron.ENOTSUP
    plan.close()
