"""Thin ctypes binding of libphikron (the C ABI in include/phikron.h).

Argument marshalling only: every step of phi_l(-tau*A)v runs inside the CUDA library.
Device buffers are torch CUDA tensors (PyTorch supplies device memory and streams); the
library receives their raw pointers.  If the shared library is missing or cannot be
loaded this module raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# the bounds-checked build (every kernel access range-checked; slow) when PHIKRON_CHECKED is 1
CHECKED = os.environ.get("PHIKRON_CHECKED") == "1"
LIB_PATH = os.path.join(HERE, "libphikron_checked.so" if CHECKED else "libphikron.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOTCONVERGED, ENOTSUP, EBOUNDS = 0, -1, -2, -3, -4, -5, -6, -7
QUAD_GAUSS, QUAD_CC, QUAD_CC_ADAPTIVE = 0, 1, 2
PREC_FP64, PREC_OZAKI_BF16 = 0, 2
SELECT_PAPER, SELECT_MLP = 0, 1
SELECTOR_USED = {0: "algorithm5", 1: "network", 2: "network+m", 3: "fallback"}

_ERRNAMES = {EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA", ETIMEOUT: "ETIMEOUT",
             ENOTCONVERGED: "ENOTCONVERGED", ENOTSUP: "ENOTSUP", EBOUNDS: "EBOUNDS"}


class PhikronError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"phikron {_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class Opts(C.Structure):
    _fields_ = [("quad", C.c_int), ("precision", C.c_int), ("selector", C.c_int),
                ("force_s", C.c_int), ("force_m", C.c_int), ("alpha", C.c_double),
                ("beta", C.c_double), ("device", C.c_int), ("max_rhs", C.c_int), ("slices", C.c_int),
                ("half_step", C.c_int), ("skip_phi0", C.c_int), ("wait_us", C.c_int)]


class Info(C.Structure):
    _fields_ = [("dims", C.c_int), ("n", C.c_int * 6), ("N", C.c_int64), ("l_max", C.c_int),
                ("s", C.c_int), ("m", C.c_int), ("cost", C.c_int), ("actions", C.c_int),
                ("alpha", C.c_double), ("log10_bound", C.c_double), ("precision", C.c_int),
                ("quad", C.c_int), ("selector_used", C.c_int), ("unique_factors", C.c_int),
                ("device_bytes", C.c_size_t), ("slices", C.c_int), ("adaptive_nodes", C.c_int),
                ("adaptive_err", C.c_double), ("fused_weights", C.c_int)]


class Profile(C.Structure):
    _fields_ = [("ms", C.c_double * 6), ("launches", C.c_longlong * 6), ("timed_launches", C.c_longlong)]


KERNEL_CLASSES = ("gemm_f64", "weighted_sum", "squaring", "tc_mode", "convert", "other")


class ErkInfo(C.Structure):
    _fields_ = [("method", C.c_int), ("nplans", C.c_int), ("applies_per_step", C.c_int),
                ("c", C.c_double * 3), ("s", C.c_int * 3), ("m", C.c_int * 3), ("actions", C.c_int * 3)]


class BatchInfo(C.Structure):
    _fields_ = [("units", C.c_int), ("launches", C.c_int), ("mode_jobs", C.c_longlong), ("graph", C.c_int),
                ("k_chunk", C.c_int), ("big_first", C.c_int), ("grid", C.c_int), ("candidates", C.c_int),
                ("tuned", C.c_int), ("best_ms", C.c_double), ("device_bytes", C.c_size_t), ("ws_kernel", C.c_int)]

_lib = None

_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int)

# name -> (restype, argtypes); every symbol declared in include/phikron.h
SIGNATURES = {
    "phikron_opts_default": (None, [C.POINTER(Opts)]),
    "phikron_plan": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(_DP), _IP, C.c_double,
                               C.c_int, C.c_double, C.POINTER(Opts)]),
    "phikron_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "phikron_apply_many": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "phikron_apply_host": (C.c_int, [C.c_void_p, _DP, _DP, C.c_void_p]),
    "phikron_apply_host_many": (C.c_int, [C.c_void_p, _DP, _DP, C.c_int, C.c_void_p]),
    "phikron_plan_info": (C.c_int, [C.c_void_p, C.POINTER(Info)]),
    "phikron_plan_nodes": (C.c_int, [C.c_void_p, _DP, _DP]),
    "phikron_destroy": (None, [C.c_void_p]),
    "phikron_check_status": (C.c_int, [C.c_void_p]),
    "phikron_last_error": (C.c_char_p, []),
    "phikron_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_void_p), C.c_int,
                                       C.c_int, C.c_int]),
    "phikron_batch_apply": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_void_p]),
    "phikron_batch_get_info": (C.c_int, [C.c_void_p, C.POINTER(BatchInfo)]),
    "phikron_batch_check_status": (C.c_int, [C.c_void_p]),
    "phikron_batch_destroy": (None, [C.c_void_p]),
    "phikron_apply_combo": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "phikron_erk_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.POINTER(_DP), C.POINTER(C.c_int),
                                     C.c_double, C.c_double, C.c_int, C.POINTER(Opts)]),
    "phikron_erk_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "phikron_erk_get_info": (C.c_int, [C.c_void_p, C.POINTER(ErkInfo)]),
    "phikron_erk_check_status": (C.c_int, [C.c_void_p]),
    "phikron_erk_profile_begin": (C.c_int, [C.c_void_p, C.c_int]),
    "phikron_batch_profile_begin": (C.c_int, [C.c_void_p, C.c_int]),
    "phikron_batch_profile_end": (C.c_int, [C.c_void_p, C.POINTER(Profile)]),
    "phikron_erk_profile_end": (C.c_int, [C.c_void_p, C.POINTER(Profile)]),
    "phikron_erk_destroy": (None, [C.c_void_p]),
    "phikron_selector_features": (C.c_int, [C.c_int, _IP, _DP, C.c_int, C.c_double, C.POINTER(C.c_float)]),
    "phikron_selector_criterion": (C.c_int, [C.c_double, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, _DP]),
    "phikron_selector_search": (C.c_int, [C.c_int, _DP, _DP, _IP, _DP, C.c_int, C.c_int, _IP, _IP, _IP]),
    "phikron_selector_param_count": (C.c_int, []),
    "phikron_selector_set_model": (C.c_int, [C.POINTER(C.c_float), C.c_int]),
    "phikron_selector_get_model": (C.c_int, [C.POINTER(C.c_float), C.c_int]),
    "phikron_selector_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_void_p]),
    "phikron_selector_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                        C.c_void_p, C.c_void_p]),
    "phikron_selector_train": (C.c_int, [C.POINTER(C.c_float), _IP, _IP, C.c_int, C.c_int, C.c_int, C.c_float,
                                         C.c_uint, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                         C.POINTER(C.c_float)]),
    "phikron_profile_begin": (C.c_int, [C.c_void_p, C.c_int]),
    "phikron_profile_end": (C.c_int, [C.c_void_p, C.POINTER(Profile)]),
    "phikron_log_quaderr": (C.c_int, [C.c_double, C.c_int, C.c_double, C.c_double, C.c_int, _DP]),
    "phikron_quadnodes": (C.c_int, [C.c_double, C.c_int, C.c_double, C.c_double, C.c_int, _IP]),
    "phikron_setup_quadrature": (C.c_int, [C.c_double, C.c_int, C.c_double, C.c_double, C.c_int,
                                           _IP, _IP, _IP]),
    "phikron_gauss_legendre": (C.c_int, [C.c_int, _DP, _DP]),
    "phikron_clenshaw_curtis": (C.c_int, [C.c_int, _DP, _DP]),
    "phikron_expm_workspace_bytes": (C.c_size_t, [C.c_int, C.c_int]),
    "phikron_live_device_buffers": (C.c_longlong, []),
    "phikron_expm_batched": (C.c_int, [C.c_int, C.c_int, C.c_void_p, _DP, _DP, C.c_void_p,
                                       C.c_void_p, C.c_void_p]),
    "phikron_kron_apply_f64": (C.c_int, [C.c_int, _IP, C.POINTER(C.c_void_p), C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p]),
    "phikron_noalloc_max_elements": (C.c_longlong, []),
    "phikron_checked": (C.c_int, []),
    "phikron_checked_violation": (C.c_int, [C.POINTER(C.c_int), C.POINTER(C.c_ulonglong),
                                            C.POINTER(C.c_ulonglong), C.POINTER(C.c_int)]),
    "phikron_checked_site_name": (C.c_char_p, [C.c_int]),
    "phikron_kron_apply_f64_noalloc": (C.c_int, [C.c_int, _IP, C.POINTER(C.c_void_p), C.c_void_p,
                                                 C.c_void_p, C.c_void_p]),
}


def lib():
    """Loads libphikron.so (libphikron_checked.so with PHIKRON_CHECKED=1; raises if it is
    absent: build it with paper_2211_00696_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{os.path.basename(LIB_PATH)} not built at {LIB_PATH}; run "
                              "`python -m paper_2211_00696_gb300.build`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int):
    if rc != OK:
        raise PhikronError(rc, lib().phikron_last_error().decode())


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def _stream_ptr(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


# ----------------------------------------------------------------------------- planner (host)

def log_quaderr(n: float, p: int, alpha: float, beta: float = 1.0, rule: int = QUAD_GAUSS) -> float:
    out = C.c_double()
    _check(lib().phikron_log_quaderr(n, p, alpha, beta, rule, C.byref(out)))
    return out.value


def quadnodes(eps: float, p: int, alpha: float, beta: float = 1.0, rule: int = QUAD_GAUSS) -> int:
    out = C.c_int()
    _check(lib().phikron_quadnodes(eps, p, alpha, beta, rule, C.byref(out)))
    return out.value


def setup_quadrature(eps: float, p: int, alpha: float, beta: float = 1.0, rule: int = QUAD_GAUSS):
    s, m, c = C.c_int(), C.c_int(), C.c_int()
    _check(lib().phikron_setup_quadrature(eps, p, alpha, beta, rule, C.byref(s), C.byref(m), C.byref(c)))
    return s.value, m.value, c.value


def gauss_legendre(m: int):
    x, w = np.zeros(m), np.zeros(m)
    _check(lib().phikron_gauss_legendre(m, _dp(x), _dp(w)))
    return x, w


def clenshaw_curtis(n: int):
    x, w = np.zeros(n + 1), np.zeros(n + 1)
    _check(lib().phikron_clenshaw_curtis(n, _dp(x), _dp(w)))
    return x, w


# ----------------------------------------------------------------------------- plans

class Plan:
    """phikron_plan_t owner.  ``factors``: list of 1 to 6 square float64 arrays (host), one per
    dimension of the Kronecker sum."""

    def __init__(self, factors, tau: float, l_max: int, tol: float, *, precision: int = PREC_FP64,
                 quad: int = QUAD_GAUSS, force_s: int = -1, force_m: int = -1, alpha: float = 0.0,
                 beta: float = 0.0, device: int = -1, max_rhs: int = 1, slices: int = 0,
                 half_step: bool = False, selector: int = SELECT_PAPER, skip_phi0: bool = False,
                 wait_us: int = 0):
        L = lib()
        self._h = C.c_void_p()
        facs = [np.ascontiguousarray(a, dtype=np.float64) for a in factors]
        self._facs = facs
        ptrs = (_DP * len(facs))(*[_dp(a) for a in facs])
        ns = (C.c_int * len(facs))(*[a.shape[0] for a in facs])
        for a in facs:
            if a.ndim != 2 or a.shape[0] != a.shape[1]:
                raise ValueError("factors must be square matrices")
        o = Opts()
        L.phikron_opts_default(C.byref(o))
        o.quad, o.precision, o.force_s, o.force_m = quad, precision, force_s, force_m
        o.alpha, o.beta, o.device, o.max_rhs, o.slices = alpha, beta, device, max_rhs, slices
        o.half_step = 1 if half_step else 0
        o.skip_phi0 = 1 if skip_phi0 else 0
        o.selector = selector
        o.wait_us = wait_us
        _check(L.phikron_plan(C.byref(self._h), len(facs), ptrs, ns, tau, l_max, tol, C.byref(o)))
        self.shape = tuple(a.shape[0] for a in facs)
        self.N = int(np.prod(self.shape))
        self.l_max = l_max
        self.max_rhs = max_rhs
        self.nout = (l_max + 1) * (2 if half_step else 1)

    def apply_combo(self, B, Out=None, stream=None):
        """sum_j phi_j(-tau A) b_j for B of shape (l_max, N) (CUDA float64); plans with s = 0."""
        import torch
        if Out is None:
            Out = torch.empty(self.N, dtype=torch.float64, device=B.device)
        _check(lib().phikron_apply_combo(self._h, B.data_ptr(), Out.data_ptr(), _stream_ptr(stream)))
        return Out

    def info(self) -> dict:
        inf = Info()
        _check(lib().phikron_plan_info(self._h, C.byref(inf)))
        return {k: (list(getattr(inf, k)) if k == "n" else getattr(inf, k)) for k, _ in Info._fields_}

    def nodes(self):
        m = self.info()["m"]
        x, w = np.zeros(max(m, 1)), np.zeros(max(m, 1))
        _check(lib().phikron_plan_nodes(self._h, _dp(x), _dp(w)))
        return x[:m], w[:m]

    def apply(self, V, Out=None, stream=None):
        """V: CUDA float64 tensor with N entries; returns Out of shape (l_max+1, N)."""
        import torch
        if V.dtype != torch.float64 or not V.is_cuda or not V.is_contiguous() or V.numel() != self.N:
            raise ValueError("V must be a contiguous CUDA float64 tensor with N entries")
        if Out is None:
            Out = torch.empty((self.nout, self.N), dtype=torch.float64, device=V.device)
        _check(lib().phikron_apply(self._h, V.data_ptr(), Out.data_ptr(), _stream_ptr(stream)))
        return Out

    def apply_many(self, V, Out=None, stream=None):
        """V: (nrhs, N) CUDA float64; returns (nrhs, l_max+1, N)."""
        import torch
        nrhs = V.shape[0]
        if Out is None:
            Out = torch.empty((nrhs, self.nout, self.N), dtype=torch.float64, device=V.device)
        _check(lib().phikron_apply_many(self._h, nrhs, V.data_ptr(), Out.data_ptr(), _stream_ptr(stream)))
        return Out

    def apply_host(self, v: np.ndarray, out: np.ndarray | None = None, stream=None) -> np.ndarray:
        """Host-memory apply (copies in, applies, copies out; synchronous)."""
        v = np.ascontiguousarray(v, dtype=np.float64).ravel()
        if out is None:
            out = np.empty((self.nout, self.N))
        st = 0 if stream is None else _stream_ptr(stream)
        _check(lib().phikron_apply_host(self._h, _dp(v), _dp(out), C.c_void_p(st)))
        return out

    def apply_host_ptr(self, v_ptr: int, out_ptr: int, stream=None):
        """Host-memory apply on raw (e.g. pinned torch) host pointers."""
        st = 0 if stream is None else _stream_ptr(stream)
        _check(lib().phikron_apply_host(self._h, C.cast(C.c_void_p(v_ptr), _DP),
                                        C.cast(C.c_void_p(out_ptr), _DP), C.c_void_p(st)))

    def apply_host_many(self, v: np.ndarray, out: np.ndarray | None = None, stream=None) -> np.ndarray:
        """Host-memory applies of count vectors (v: (count, N)) with pipelined transfers;
        returns (count, l_max+1, N).  Pinned buffers (apply_host_many_ptr) overlap the copies."""
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, self.N)
        count = v.shape[0]
        if out is None:
            out = np.empty((count, self.nout, self.N))
        st = 0 if stream is None else _stream_ptr(stream)
        _check(lib().phikron_apply_host_many(self._h, _dp(v), _dp(out), count, C.c_void_p(st)))
        return out

    def apply_host_many_ptr(self, v_ptr: int, out_ptr: int, count: int, stream=None):
        """apply_host_many on raw (e.g. pinned torch) host pointers."""
        st = 0 if stream is None else _stream_ptr(stream)
        _check(lib().phikron_apply_host_many(self._h, C.cast(C.c_void_p(v_ptr), _DP),
                                             C.cast(C.c_void_p(out_ptr), _DP), count, C.c_void_p(st)))

    def check_status(self):
        """Raises PhikronError(ETIMEOUT) if a bounded device wait of an earlier apply expired."""
        _check(lib().phikron_check_status(self._h))

    def profile_begin(self, max_timed: int = 0):
        """Count (and, if max_timed > 0, event-time) every kernel the applies launch."""
        _check(lib().phikron_profile_begin(self._h, max_timed))

    def profile_end(self) -> dict:
        pr = Profile()
        _check(lib().phikron_profile_end(self._h, C.byref(pr)))
        return {"ms": dict(zip(KERNEL_CLASSES, list(pr.ms))),
                "launches": dict(zip(KERNEL_CLASSES, list(pr.launches))),
                "timed_launches": pr.timed_launches}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().phikron_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """phikron_batch_t owner: plans x nrhs right-hand sides in grouped launches (one graph)."""

    def __init__(self, plans, nrhs: int = 1, half_step: bool = False, autotune: bool = False):
        self._plans = list(plans)
        self._h = C.c_void_p()
        arr = (C.c_void_p * len(self._plans))(*[p._h.value for p in self._plans])
        _check(lib().phikron_batch_create(C.byref(self._h), len(self._plans), arr, nrhs,
                                          1 if half_step else 0, 1 if autotune else 0))
        self.nrhs = nrhs
        self.half_step = half_step

    def apply(self, V, Out=None, stream=None):
        """V: list of CUDA float64 tensors (nrhs, N_i); returns list of (nrhs, nout, N_i)."""
        import torch
        if Out is None:
            Out = [torch.empty((self.nrhs, p.nout, p.N), dtype=torch.float64, device=v.device)
                   for p, v in zip(self._plans, V)]
        vp = (C.c_void_p * len(V))(*[v.data_ptr() for v in V])
        op = (C.c_void_p * len(Out))(*[o.data_ptr() for o in Out])
        _check(lib().phikron_batch_apply(self._h, vp, op, _stream_ptr(stream)))
        return Out

    def info(self) -> dict:
        inf = BatchInfo()
        _check(lib().phikron_batch_get_info(self._h, C.byref(inf)))
        return {k: getattr(inf, k) for k, _ in BatchInfo._fields_}

    def profile_begin(self, max_timed: int = 0):
        """Count (and, if max_timed > 0, event-time) the kernels of the following applies."""
        _check(lib().phikron_batch_profile_begin(self._h, max_timed))

    def profile_end(self) -> dict:
        pr = Profile()
        _check(lib().phikron_batch_profile_end(self._h, C.byref(pr)))
        return {"ms": dict(zip(KERNEL_CLASSES, list(pr.ms))),
                "launches": dict(zip(KERNEL_CLASSES, list(pr.launches))),
                "timed_launches": pr.timed_launches}

    def check_status(self):
        _check(lib().phikron_batch_check_status(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().phikron_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


ERK_EULER, ERK_RK2, ERK_RK3 = 1, 2, 3
NONLIN_NONE, NONLIN_ALLEN_CAHN = 0, 1


class Integrator:
    """phikron_erk_t owner: exponential Euler / RK2 (c2 = 1/2) / RK3 (c2 = 1/3, c3 = 2/3) for
    u' + A u = f(u), A the Kronecker sum of ``factors``; every phi-action runs in this library."""

    def __init__(self, factors, tau: float, method: int, tol: float, *, nonlinearity: int = NONLIN_ALLEN_CAHN,
                 precision: int = PREC_FP64, slices: int = 0, device: int = -1):
        L = lib()
        facs = [np.ascontiguousarray(a, dtype=np.float64) for a in factors]
        self._facs = facs
        ptrs = (_DP * len(facs))(*[_dp(a) for a in facs])
        ns = (C.c_int * len(facs))(*[a.shape[0] for a in facs])
        o = Opts()
        L.phikron_opts_default(C.byref(o))
        o.precision, o.slices, o.device = precision, slices, device
        self._h = C.c_void_p()
        _check(L.phikron_erk_create(C.byref(self._h), method, len(facs), ptrs, ns, tau, tol, nonlinearity,
                                    C.byref(o)))
        self.N = int(np.prod([a.shape[0] for a in facs]))

    def step(self, U, nsteps: int = 1, stream=None):
        """Advances U (CUDA float64 tensor with N elements, updated in place) by nsteps steps."""
        _check(lib().phikron_erk_step(self._h, U.data_ptr(), nsteps, _stream_ptr(stream)))
        return U

    def info(self) -> dict:
        inf = ErkInfo()
        _check(lib().phikron_erk_get_info(self._h, C.byref(inf)))
        return {k: (list(getattr(inf, k)) if k in ("c", "s", "m", "actions") else getattr(inf, k))
                for k, _ in ErkInfo._fields_}

    def profile_begin(self, max_timed: int = 0):
        """Count (and, if max_timed > 0, event-time) the kernels of the following steps."""
        _check(lib().phikron_erk_profile_begin(self._h, max_timed))

    def profile_end(self) -> dict:
        pr = Profile()
        _check(lib().phikron_erk_profile_end(self._h, C.byref(pr)))
        return {"ms": dict(zip(KERNEL_CLASSES, list(pr.ms))),
                "launches": dict(zip(KERNEL_CLASSES, list(pr.launches))),
                "timed_launches": pr.timed_launches}

    def check_status(self):
        _check(lib().phikron_erk_check_status(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().phikron_erk_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------- kernels alone

def expm_batched(A, scale, stream=None):
    """E[b] = exp(scale[b] * A[b]); A: (count, n, n) CUDA float64 tensor; scale: host floats."""
    import torch
    count, n, _ = A.shape
    A = A.contiguous()
    sc = np.ascontiguousarray(scale, dtype=np.float64)
    E = torch.empty_like(A)
    ws = torch.empty(int(lib().phikron_expm_workspace_bytes(count, n)) // 8 + 1, dtype=torch.float64,
                     device=A.device)
    # norms1 = NULL: the library takes ||A[b]||_1 itself (synchronous)
    _check(lib().phikron_expm_batched(count, n, A.data_ptr(), _dp(sc), None, E.data_ptr(),
                                      ws.data_ptr(), _stream_ptr(stream)))
    return E


def kron_apply_f64(mats, V, stream=None):
    """(mats[0] (x) ... ) V for CUDA float64 tensors (mode products in float64)."""
    import torch
    ns = (C.c_int * len(mats))(*[m.shape[0] for m in mats])
    ptrs = (C.c_void_p * len(mats))(*[m.contiguous().data_ptr() for m in mats])
    out = torch.empty_like(V)
    work = torch.empty_like(V)
    _check(lib().phikron_kron_apply_f64(len(mats), ns, ptrs, V.data_ptr(), out.data_ptr(),
                                        work.data_ptr(), _stream_ptr(stream)))
    return out


def checked_violation() -> dict:
    """The bounds-checked build's first recorded out-of-range access since the last read
    (site 0: none) and the number of them; reading clears the record."""
    site, cnt = C.c_int(), C.c_int()
    addr, nb = C.c_ulonglong(), C.c_ulonglong()
    _check(lib().phikron_checked_violation(C.byref(site), C.byref(addr), C.byref(nb), C.byref(cnt)))
    return {"site": site.value, "name": lib().phikron_checked_site_name(site.value).decode(),
            "addr": addr.value, "bytes": nb.value, "count": cnt.value}

