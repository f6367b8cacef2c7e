"""Host-buffer entry points through the C ABI: the pipelined phikron_apply_host_many (transfers
of neighbouring vectors overlap the apply) returns, vector by vector, bitwise the results of
phikron_apply on device buffers and of the synchronous phikron_apply_host, for the float64 and
the mixed path, pinned and pageable host memory, one vector and several (both staging sets
reused), and with half-step outputs."""
import numpy as np
import pytest

import workloads as W
from oracle import phi as P

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _pk():
    import paper_2211_00696_gb300 as pk
    return pk


def _plan(prec, **kw):
    pk = _pk()
    shape = (32, 48, 64)
    fac = [W.convdiff_factor(n) for n in shape]
    plan = pk.Plan(fac, 1e-2, 3, 1e-10, precision=pk.PREC_FP64 if prec == "fp64" else pk.PREC_OZAKI_BF16, **kw)
    return plan, fac, shape


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("count", [1, 5])
def test_pipelined_host_applies_match_device_applies(prec, count):
    plan, fac, shape = _plan(prec)
    N = int(np.prod(shape))
    V = np.stack([W.uniform_vector(shape, 30 + j) for j in range(count)])
    vh = torch.from_numpy(V).pin_memory()
    oh = torch.full((count, plan.nout, N), float("nan"), dtype=torch.float64).pin_memory()
    plan.apply_host_many_ptr(vh.data_ptr(), oh.data_ptr(), count)
    got = oh.numpy()
    for j in range(count):
        ref = plan.apply(torch.from_numpy(V[j]).cuda()).cpu().numpy()
        assert np.array_equal(got[j], ref), (prec, j)
        assert np.array_equal(got[j], plan.apply_host(V[j])), (prec, j)
    plan.check_status()
    # pageable buffers through the same entry point
    out = plan.apply_host_many(V)
    assert np.array_equal(out, got)
    # and against the definition for the last vector
    exact = P.phi_sparse(fac, 1e-2, V[-1], 3)
    for l in range(4):
        assert P.rel_err_2(got[-1][l], exact[l]) <= 1e-9


def test_pipelined_host_applies_half_step_layout():
    plan, fac, shape = _plan("mixed", half_step=True)   # half-step outputs: mixed path only
    N = int(np.prod(shape))
    V = np.stack([W.uniform_vector(shape, 40 + j) for j in range(3)])
    out = plan.apply_host_many(V)
    assert out.shape == (3, 8, N)
    for j in range(3):
        ref = plan.apply(torch.from_numpy(V[j]).cuda()).cpu().numpy()
        assert np.array_equal(out[j], ref.reshape(8, N))


def test_pipelined_host_applies_reject_bad_count():
    pk = _pk()
    plan, _, shape = _plan("fp64")
    v = np.zeros((1, int(np.prod(shape))))
    o = np.zeros((1, plan.nout, v.shape[1]))
    from paper_2211_00696_gb300 import phikron as B
    import ctypes as C
    rc = pk.lib().phikron_apply_host_many(plan._h, v.ctypes.data_as(B._DP), o.ctypes.data_as(B._DP), 0, None)
    assert rc == B.EINVAL
