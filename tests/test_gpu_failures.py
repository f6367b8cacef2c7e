"""Failure paths, made on the host or through status codes (no test here faults, traps or hangs
the GPU):

* allocation failure: PHIKRON_FAIL_ALLOC_AFTER = k refuses the library's allocations after the
  first k; every k up to the count a create call needs gives PHIKRON_ENOMEM, and the number of
  device buffers the library holds (phikron_live_device_buffers) is back at its previous value
  after each failure, for a mixed plan (its launch sequence included), a batch, an integrator;
* a bounded device wait that expires: a plan whose wait limit is 1 microsecond (far shorter
  than a tile of tensor-core work) makes the kernels give up; phikron_check_status reports
  PHIKRON_ETIMEOUT, and a plan with the default limit, made afterwards in the same context,
  gives correct results.
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


def _live():
    return int(_pk().lib().phikron_live_device_buffers())


def _fail_until_success(monkeypatch, make):
    """Calls make() with PHIKRON_FAIL_ALLOC_AFTER = 0, 1, 2, ... until it succeeds; returns the
    object and the number of refused attempts.  Each refusal must be ENOMEM and leak nothing."""
    pk = _pk()
    base = _live()
    for k in range(0, 400):
        monkeypatch.setenv("PHIKRON_FAIL_ALLOC_AFTER", str(k))
        try:
            obj = make()
        except pk.PhikronError as e:
            assert e.code == pk.phikron.ENOMEM, (k, str(e))
            assert _live() == base, (k, _live(), base)
            continue
        finally:
            monkeypatch.delenv("PHIKRON_FAIL_ALLOC_AFTER", raising=False)
        return obj, k
    raise AssertionError("never succeeded")


def test_plan_allocation_failures(monkeypatch):
    pk = _pk()
    shape = (32, 48, 64)
    fac = [W.convdiff_factor(n) for n in shape]
    v = W.uniform_vector(shape, 3)
    warm = pk.Plan(fac, 1e-2, 3, 1e-9, precision=pk.PREC_OZAKI_BF16, slices=4)   # module loading
    warm.close()
    base = _live()
    plan, refused = _fail_until_success(
        monkeypatch, lambda: pk.Plan(fac, 1e-2, 3, 1e-9, precision=pk.PREC_OZAKI_BF16, slices=4))
    assert refused >= 10          # host object, expm staging, work buffers, sequence tables ...
    out = plan.apply(torch.from_numpy(v).cuda()).cpu().numpy()
    plan.check_status()
    ref = pk.Plan(fac, 1e-2, 3, 1e-9, force_s=plan.info()["s"], force_m=plan.info()["m"])
    exp = ref.apply(torch.from_numpy(v).cuda()).cpu().numpy()
    for l in range(4):
        assert P.rel_err_2(out[l], exp[l]) <= 5e-8
    plan.close()
    ref.close()
    assert _live() == base


def test_batch_and_integrator_allocation_failures(monkeypatch):
    pk = _pk()
    plans = [pk.Plan([W.laplacian_factor(n, 0.5) for n in shape], 1e-3, 3, 1e-6, precision=pk.PREC_OZAKI_BF16,
                     slices=3, half_step=True) for shape in ((32, 32, 48), (64, 32, 16))]
    base = _live()
    batch, refused = _fail_until_success(monkeypatch, lambda: pk.Batch(plans, nrhs=2, half_step=True))
    assert refused >= 3
    batch.close()
    assert _live() == base
    a = W.periodic_diffusion_factor(64, 1e-3)
    it, refused = _fail_until_success(monkeypatch, lambda: pk.Integrator([a, a], 1e-2, pk.ERK_RK2, 1e-8,
                                                                         precision=pk.PREC_OZAKI_BF16))
    assert refused >= 3
    it.close()
    assert _live() == base
    for p in plans:
        p.close()


def test_expired_wait_reports_timeout_and_next_plan_is_correct():
    pk = _pk()
    shape = (64, 160, 96)
    fac = [W.convdiff_factor(n) for n in shape]
    v = W.uniform_vector(shape, 11)
    V = torch.from_numpy(v).cuda()
    short = pk.Plan(fac, 1e-2, 3, 1e-9, precision=pk.PREC_OZAKI_BF16, slices=4, wait_us=1)
    short.apply(V)
    with pytest.raises(pk.PhikronError) as e:
        short.check_status()
    assert e.value.code == pk.phikron.ETIMEOUT
    short.check_status()           # the status was cleared by the first check
    short.close()
    good = pk.Plan(fac, 1e-2, 3, 1e-9, precision=pk.PREC_OZAKI_BF16, slices=4)
    out = good.apply(V).cpu().numpy()
    good.check_status()
    info = good.info()
    ref = pk.Plan(fac, 1e-2, 3, 1e-9, force_s=info["s"], force_m=info["m"])
    exp = ref.apply(V).cpu().numpy()
    for l in range(4):
        assert P.rel_err_2(out[l], exp[l]) <= 5e-8, l
    good.close()
    ref.close()
