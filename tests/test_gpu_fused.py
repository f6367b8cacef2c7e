"""The fused node-weight pass (Algorithm 1's weighted sums y_j = sum_k c_{j,k} T_k formed in the
epilogue of the last mode pass of the node phase, so that no node product T_k is written to
device memory) against the separate pass pair it replaces.

The fused epilogue forms every T_k with the same operations as the separate mode kernel and
adds c_{j,k} T_k in the same order, with the same round-to-nearest float-float operations, as
the separate weighted-sum kernel: the outputs must be equal bit for bit.  Plans are built
twice from the same inputs, once with the fused pass (PHIKRON_FUSED_WEIGHTS=1) and once
without it, with the same (s, m).  The cases cover every digit-slice count, 1 to
4 weighted outputs, s = 0 (the weighted sums are the float64 outputs) and s > 0 (they feed the
squaring steps), the half-step outputs, phi_0 skipped, a contracted size below 128 with a half
chunk (n = 48, 80), ragged fiber tiles (B0 not a multiple of 32), several tiles per CTA, and
2D and 4D Kronecker sums; plus the cases that keep the separate pass.
"""
import numpy as np
import pytest

import workloads as W
from oracle import phi as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _pk():
    import paper_2211_00696_gb300 as pk
    return pk


def _pair(monkeypatch, fac, tau, p, tol, v, **kw):
    pk = _pk()
    monkeypatch.setenv("PHIKRON_FUSED_WEIGHTS", "1")
    fused = pk.Plan(fac, tau, p, tol, precision=pk.PREC_OZAKI_BF16, **kw)
    info = fused.info()
    monkeypatch.setenv("PHIKRON_FUSED_WEIGHTS", "0")
    kw2 = dict(kw)
    kw2["force_s"], kw2["force_m"] = info["s"], info["m"]
    sep = pk.Plan(fac, tau, p, tol, precision=pk.PREC_OZAKI_BF16, **kw2)
    monkeypatch.delenv("PHIKRON_FUSED_WEIGHTS")
    V = torch.from_numpy(v).cuda()
    a = fused.apply(V).cpu().numpy()
    b = sep.apply(V).cpu().numpy()
    fused.check_status()
    sep.check_status()
    out = (a, b, info, sep.info())
    fused.close()
    sep.close()
    return out


CASES = [
    # shape, tau, l_max, tol, slices, extra options
    ((32, 48, 64), 1e-2, 3, 1e-10, 5, {}),
    ((64, 160, 96), 1e-2, 3, 1e-9, 4, {}),          # 15360 fibers: 480 tiles, several per CTA
    ((48, 32, 48), 1e-2, 2, 1e-6, 3, {}),           # n = 48: a half K chunk; 1536 fibers
    ((16, 17 * 16, 80), 5e-3, 4, 1e-10, 6, {}),     # n = 80, 4352 fibers, p = 4
    ((48, 112), 1e-2, 1, 1e-8, 4, {}),              # 2D, p = 1, 48 fibers (a ragged tile of 16)
    ((16, 32), 1e-2, 2, 1e-8, 5, {}),               # 2D, n = 32 (one K chunk), a single tile of 16 fibers
    ((16, 16, 16, 32), 1e-2, 3, 1e-9, 4, {}),       # 4D
    ((32, 48, 64), 1e-6, 3, 1e-9, 4, {}),           # s = 0: weighted sums are the float64 outputs
    ((32, 48, 64), 1e-2, 3, 1e-9, 4, {"half_step": True}),
    ((32, 48, 64), 1e-7, 2, 1e-9, 4, {"half_step": True}),   # half_step forces s = 1: y_j copied at tau/2
    ((32, 48, 64), 1e-2, 3, 1e-9, 4, {"skip_phi0": True}),
]


@pytest.mark.parametrize("shape,tau,p,tol,slices,kw", CASES)
def test_fused_pass_is_bitwise_the_separate_passes(monkeypatch, shape, tau, p, tol, slices, kw):
    fac = [W.convdiff_factor(n) for n in shape]
    v = W.uniform_vector(shape, 41)
    a, b, fi, si = _pair(monkeypatch, fac, tau, p, tol, v, slices=slices, **kw)
    assert fi["fused_weights"] == 1 and si["fused_weights"] == 0
    assert (fi["s"], fi["m"]) == (si["s"], si["m"])
    if kw.get("skip_phi0"):
        a, b = a[1:], b[1:]          # phi_0 slots are left untouched
    assert np.all(np.isfinite(a))
    if not np.array_equal(a, b):
        d = np.max(np.abs(a - b)) / np.max(np.abs(b))
        pytest.fail(f"fused differs from separate passes: max rel diff {d:.3e}")


def test_fused_pass_matches_the_definition(monkeypatch):
    """The fused path against the sparse augmented-matrix oracle (O3) on a small nonsymmetric
    3D operator with three different factors."""
    pk = _pk()
    monkeypatch.setenv("PHIKRON_FUSED_WEIGHTS", "1")
    shape = (16, 32, 48)
    fac = [W.convdiff_factor(shape[0]), W.laplacian_factor(shape[1], 0.5), W.convdiff_factor(shape[2])]
    v = W.uniform_vector(shape, 5)
    plan = pk.Plan(fac, 1e-2, 3, 1e-10, precision=pk.PREC_OZAKI_BF16, slices=6)
    assert plan.info()["fused_weights"] == 1
    out = plan.apply(torch.from_numpy(v).cuda()).cpu().numpy()
    plan.check_status()
    exact = P.phi_sparse(fac, 1e-2, v, 3)
    for l in range(4):
        assert P.rel_err_2(out[l], exact[l]) <= 1e-11, l


def test_cases_that_keep_the_separate_pass(monkeypatch):
    pk = _pk()
    monkeypatch.setenv("PHIKRON_FUSED_WEIGHTS", "1")
    # last factor above 128 rows, l_max above 4, one factor, l_max = 0, and the float64 path
    for fac, p in (([W.laplacian_factor(32), W.laplacian_factor(144)], 2),
                   ([W.laplacian_factor(32), W.laplacian_factor(32)], 5),
                   ([W.laplacian_factor(64)], 2),
                   ([W.laplacian_factor(32), W.laplacian_factor(32)], 0)):
        plan = pk.Plan(fac, 1e-3, p, 1e-8, precision=pk.PREC_OZAKI_BF16)
        assert plan.info()["fused_weights"] == 0
        plan.close()
    plan = pk.Plan([W.laplacian_factor(32)] * 2, 1e-3, 2, 1e-8)
    assert plan.info()["fused_weights"] == 0
    plan.close()
