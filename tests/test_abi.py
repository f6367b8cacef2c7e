"""The C-ABI library loads on a machine without a GPU, exports every symbol the header
declares, and its host-only planner agrees exactly with the oracle planner."""
import os
import re

import numpy as np
import pytest

import paper_2211_00696_gb300 as pk
from paper_2211_00696_gb300 import phikron as B
from oracle import planner as PL

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(phikron_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    L = pk.lib()
    declared = _declared_functions()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(L, name), name
    assert declared <= set(B.SIGNATURES), declared - set(B.SIGNATURES)


def test_checked_library_exports_every_declared_symbol():
    """The bounds-checked variant (built by the same build step) exports the same C ABI and
    reports itself; its record reads empty without any device work."""
    import ctypes as C
    from paper_2211_00696_gb300 import build as BLD
    path = BLD.CHECKED.lib
    assert os.path.exists(path), path
    L = C.CDLL(path)
    for name in _declared_functions():
        assert hasattr(L, name), name
    L.phikron_checked.restype = C.c_int
    assert L.phikron_checked() == 1
    assert pk.lib().phikron_checked() == 0
    site, cnt = C.c_int(-1), C.c_int(-1)
    addr, nb = C.c_ulonglong(1), C.c_ulonglong(1)
    for lib in (L, pk.lib()):
        assert lib.phikron_checked_violation(C.byref(site), C.byref(addr), C.byref(nb), C.byref(cnt)) == 0
        assert (site.value, cnt.value, addr.value, nb.value) == (0, 0, 0, 0)
    L.phikron_checked_site_name.restype = C.c_char_p
    assert L.phikron_checked_site_name(1) == b"mode kernel operand load"
    assert L.phikron_checked_site_name(17) == b"plan-time kernel"
    assert L.phikron_checked_site_name(18) == b"unknown"


def test_planner_matches_oracle_exactly():
    for alpha in (0.37, 2.0, 8.712, 27.7092, 384.0, 1331.2, 85196.8, 3.1e5):
        for tol in (1e-6, 1e-8, 1e-10, 1e-14):
            for p in (1, 2, 3, 7, 20):
                for rule, name in ((pk.QUAD_GAUSS, PL.GAUSS), (pk.QUAD_CC, PL.CC)):
                    assert pk.setup_quadrature(tol, p, alpha, 1.0, rule) == tuple(
                        PL.setup_quadrature(tol, p, alpha, 1.0, name)), (alpha, tol, p, rule)


def test_log_quaderr_matches_oracle():
    for n in (2, 3.5, 8, 17, 40):
        for p in (1, 3, 20):
            for alpha in (0.5, 5.0, 60.0):
                a = pk.log_quaderr(n, p, alpha)
                b = PL.log_quaderr(n, p, alpha, 1.0)
                assert abs(a - b) <= 1e-9 * max(1.0, abs(b))


def test_quadnodes_matches_oracle():
    for eps in (1e-6, 1e-10, 1e-14):
        for p in (1, 3, 20):
            for alpha in (0.1, 3.0, 48.0):
                assert pk.quadnodes(eps, p, alpha) == PL.quadnodes(eps, p, alpha, 1.0)


def test_gauss_legendre_matches_library_rule():
    for m in (1, 2, 3, 8, 9, 21, 37, 64):
        x, w = pk.gauss_legendre(m)
        xr, wr = PL.gauss_legendre_01(m)
        assert np.max(np.abs(x - xr)) <= 2e-16 * 4
        # numpy's leggauss weights drift ~1e-16*m^2 relative; the library's are pinned below
        assert np.max(np.abs(w - wr)) <= 1e-12 * np.max(wr)
        for k in range(2 * m):
            assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) <= 2e-15


def test_clenshaw_curtis_exact_on_polynomials():
    for n in (2, 6, 12, 48):
        x, w = pk.clenshaw_curtis(n)
        for k in range(n + 1):
            assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) <= 1e-14


def test_invalid_arguments_return_einval_without_gpu():
    with pytest.raises(pk.PhikronError) as e:
        pk.gauss_legendre(0)
    assert e.value.code == B.EINVAL
    with pytest.raises(pk.PhikronError) as e:
        pk.setup_quadrature(1e-10, 3, -1.0)
    assert e.value.code == B.EINVAL
    with pytest.raises(pk.PhikronError):
        pk.Plan([np.eye(3), np.eye(3)], 0.1, 25, 1e-10)      # l_max > 20
    with pytest.raises(pk.PhikronError):
        pk.Plan([np.eye(3), np.full((3, 3), np.nan)], 0.1, 2, 1e-10)
    with pytest.raises(pk.PhikronError):
        pk.Plan([np.eye(3), np.eye(3)], 0.1, 2, 0.0)          # tol <= 0
    # pipelined host applies: argument checks run before any device call
    L = pk.lib()
    assert L.phikron_apply_host_many(None, None, None, 1, None) == B.EINVAL
    # exponential integrators: argument checks run before any device call
    for bad in (dict(method=4), dict(method=1, tau=0.0), dict(method=2, nonlinearity=7)):
        kw = dict(tau=1e-2, nonlinearity=pk.NONLIN_ALLEN_CAHN)
        kw.update(bad)
        method = kw.pop("method")
        tau = kw.pop("tau")
        with pytest.raises(pk.PhikronError) as e:
            pk.Integrator([np.eye(4), np.eye(4)], tau, method, 1e-10, **kw)
        assert e.value.code == B.EINVAL


def test_kron_apply_rejects_overlapping_buffers_before_any_device_work():
    """A mode product reads its whole input while it writes its output, so V, Out (and the work
    buffer) must be separate ranges; overlapping ranges are refused before anything is launched
    (no device memory is touched: the pointers here are placeholders)."""
    import ctypes as C
    L = pk.lib()
    n = (C.c_int * 3)(4, 4, 4)           # N = 64 float64 = 512 bytes
    E = (C.c_void_p * 3)(0x10000, 0x10000, 0x10000)
    base = 0x7F0000000000
    # V == Out, and Out starting inside V
    for out in (base, base + 8 * 63):
        rc = L.phikron_kron_apply_f64_noalloc(3, n, E, base, out, None)
        assert rc == B.EINVAL and b"overlap" in L.phikron_last_error()
        rc = L.phikron_kron_apply_f64(3, n, E, base, out, base + 4096, None)
        assert rc == B.EINVAL and b"overlap" in L.phikron_last_error()
    # work overlapping V (three factors use it)
    rc = L.phikron_kron_apply_f64(3, n, E, base, base + 4096, base + 256, None)
    assert rc == B.EINVAL and b"overlap" in L.phikron_last_error()
