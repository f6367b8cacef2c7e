"""Learned (s, m) selector: training-set generation, GPU training, model I/O.

Training data: 3D reaction-diffusion Laplacians A^d = c_d (-D2) on n_d interior points
(n_d uniform in 32..256, c_d ~ logU(1e-3, 1)), tau ~ logU(1e-5, 1), l_max in 1..4,
tol in {1e-6, 1e-8, 1e-10}.  Features come from the library (the same function plans use);
labels come from the library's cost-minimising search under the measured criterion over
the Gershgorin interval [-tau sum_d 4 c_d (n_d+1)^2, 0] of -tau*A.  Everything numeric runs
in libphikron (threaded C++ search on the host, training kernels on the GPU).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .phikron import _DP, _IP, _check, lib

HERE = os.path.dirname(os.path.abspath(__file__))
MODEL_PATH = os.path.join(HERE, "selector_model.npy")
TOLS = (1e-6, 1e-8, 1e-10)


def sample_problems(count: int, seed: int):
    rng = np.random.default_rng(seed)
    n = rng.integers(32, 257, size=(count, 3))
    c = 10.0 ** rng.uniform(-3.0, 0.0, size=(count, 3))
    tau = 10.0 ** rng.uniform(-5.0, 0.0, size=count)
    p = rng.integers(1, 5, size=count)
    tol = rng.choice(TOLS, size=count)
    return n, c, tau, p, tol


def features(n, c, tau, p, tol) -> np.ndarray:
    L = lib()
    X = np.zeros((len(tau), 8), dtype=np.float32)
    for i in range(len(tau)):
        ns = (C.c_int * 3)(*[int(v) for v in n[i]])
        tn = np.ascontiguousarray([tau[i] * c[i][d] * 4.0 * (n[i][d] + 1) ** 2 for d in range(3)])
        out = (C.c_float * 8)()
        _check(L.phikron_selector_features(3, ns, tn.ctypes.data_as(_DP), int(p[i]), float(tol[i]), out))
        X[i] = np.frombuffer(out, dtype=np.float32)
    return X


def labels(n, c, tau, p, tol, npts: int = 128, nthreads: int = 0):
    zlo = np.ascontiguousarray(-tau * np.sum(4.0 * c * (n + 1.0) ** 2, axis=1))
    zhi = np.zeros_like(zlo)
    pp = np.ascontiguousarray(p, dtype=np.int32)
    tt = np.ascontiguousarray(tol, dtype=np.float64)
    s = np.zeros(len(zlo), np.int32)
    m = np.zeros(len(zlo), np.int32)
    cost = np.zeros(len(zlo), np.int32)
    _check(lib().phikron_selector_search(len(zlo), zlo.ctypes.data_as(_DP), zhi.ctypes.data_as(_DP),
                                         pp.ctypes.data_as(_IP), tt.ctypes.data_as(_DP), npts, nthreads,
                                         s.ctypes.data_as(_IP), m.ctypes.data_as(_IP), cost.ctypes.data_as(_IP)))
    return s, m, cost


def training_set(count: int, seed: int = 5):
    n, c, tau, p, tol = sample_problems(count, seed)
    X = features(n, c, tau, p, tol)
    s, m, cost = labels(n, c, tau, p, tol)
    return X, s, m, cost


def train(X, s, m, epochs: int = 150, batch: int = 512, lr: float = 2e-3, seed: int = 7):
    """Trains on the GPU with the library's kernels; the result becomes the process-wide model."""
    L = lib()
    npar = L.phikron_selector_param_count()
    Xc = np.ascontiguousarray(X, dtype=np.float32)
    sc = np.ascontiguousarray(s, dtype=np.int32)
    mc = np.ascontiguousarray(m, dtype=np.int32)
    out = (C.c_float * npar)()
    loss = C.c_float()
    _check(L.phikron_selector_train(Xc.ctypes.data_as(C.POINTER(C.c_float)), sc.ctypes.data_as(_IP),
                                    mc.ctypes.data_as(_IP), len(sc), epochs, batch, lr, seed, None, out,
                                    C.byref(loss)))
    return np.frombuffer(out, dtype=np.float32).copy(), float(loss.value)


def set_model(params: np.ndarray):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(lib().phikron_selector_set_model(p.ctypes.data_as(C.POINTER(C.c_float)), len(p)))


def load_default_model() -> bool:
    """Loads the trained model shipped with the package (if present) into the library."""
    if not os.path.exists(MODEL_PATH):
        return False
    set_model(np.load(MODEL_PATH))
    return True


if __name__ == "__main__":
    import sys
    import time
    count = int(sys.argv[1]) if len(sys.argv) > 1 else 100000
    t0 = time.time()
    X, s, m, cost = training_set(count)
    t1 = time.time()
    params, loss = train(X, s, m)
    t2 = time.time()
    np.save(MODEL_PATH, params)
    print(f"labels {t1 - t0:.1f} s, training {t2 - t1:.1f} s, final loss {loss:.4f}, saved {MODEL_PATH}")
