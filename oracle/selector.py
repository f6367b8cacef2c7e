"""Measured error criterion, cost-minimising (s, m) search and selector network in float64
-- test infrastructure only.

Criterion: for symmetric A the 2-norm error of the method equals at most the largest scalar
error over the spectrum.  The scalar method at z: Gauss-Legendre quadrature of Eq. (3) at
2^-s z (Algorithm 1), then s steps of the scalar modified squaring recurrence (Eq. (29));
compared with phi_j(z) from ``phi.phi_scalar`` for j = 1..p, maximised over Chebyshev-spaced
sample points of [zlo, zhi] (both ends included).

Search: Algorithm 5's shape with this criterion: every s from ceil(log2 max|z|)+2 (at most
20) down to 0, for each s the smallest m in 2..32 meeting tol (bisection, the criterion falls
with m), cost m + s*p; the lowest cost wins (ties keep the larger s).  The scan stops early
only when m = 32 fails below an admissible s.  Unlike Algorithm 5 it does not stop at the
first non-improving s: with this criterion the cost can plateau before it falls.

Network: 8 -> 64 -> 64 -> 52 (21 logits for s = 0..20, 31 for m = 2..32), ReLU, loss = mean
of cross-entropy(s) + cross-entropy(m); ``grads`` is the analytic backward pass.
Pinned in tests/test_oracle_selector.py (criterion dominates the true matrix error; the
search's (s, m) is minimal; gradients against finite differences).
"""
from __future__ import annotations

import math

import numpy as np

from . import planner
from .phi import phi_scalar

S_CLASSES, M_CLASSES, M_MIN = 21, 31, 2
LAYERS = ((8, 64), (64, 64), (64, S_CLASSES + M_CLASSES))


def criterion(zlo: float, zhi: float, p: int, s: int, m: int, npts: int = 128) -> float:
    x, w = planner.gauss_legendre_01(m)
    q = np.arange(npts)
    t = np.cos(np.pi * q / (npts - 1)) if npts > 1 else np.zeros(1)
    z = 0.5 * (zlo + zhi) + 0.5 * (zhi - zlo) * t
    zs = z / 2.0 ** s
    y = np.zeros((p + 1, npts))
    for k in range(m):
        e = np.exp((1.0 - x[k]) * zs)
        for j in range(1, p + 1):
            y[j] += w[k] * x[k] ** (j - 1) / math.factorial(j - 1) * e
    for t2 in range(s):
        g = np.exp(z * 2.0 ** (t2 - s))
        yn = np.zeros_like(y)
        for i in range(1, p + 1):
            acc = g * y[i]
            for j in range(1, i + 1):
                acc = acc + y[j] / math.factorial(i - j)
            yn[i] = acc / 2.0 ** i
        y = yn
    worst = 0.0
    for j in range(1, p + 1):
        worst = max(worst, float(np.max(np.abs(y[j] - phi_scalar(j, z)))))
    return worst


def search(zlo: float, zhi: float, p: int, tol: float, npts: int = 128):
    a = max(abs(zlo), abs(zhi))
    smax = int(math.ceil(math.log2(a))) + 2 if a > 0 else 0
    smax = max(0, min(20, smax))
    best = None
    for s in range(smax, -1, -1):
        if criterion(zlo, zhi, p, s, 32, npts) > tol:
            if best is not None:
                break
            continue
        lo, hi = 2, 32
        while lo < hi:
            mid = (lo + hi) // 2
            if criterion(zlo, zhi, p, s, mid, npts) <= tol:
                hi = mid
            else:
                lo = mid + 1
        cost = lo + s * p
        if best is None or cost < best[2]:
            best = (s, lo, cost)
    return best


# ----------------------------------------------------------------------------- network

def unpack(params: np.ndarray):
    out, off = [], 0
    for a, b in LAYERS:
        W = params[off:off + a * b].reshape(a, b)
        off += a * b
        bias = params[off:off + b]
        off += b
        out.append((W, bias))
    return out


def n_params() -> int:
    return sum(a * b + b for a, b in LAYERS)


def forward(params, X):
    (W1, b1), (W2, b2), (W3, b3) = unpack(np.asarray(params, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    h1 = np.maximum(X @ W1 + b1, 0.0)
    h2 = np.maximum(h1 @ W2 + b2, 0.0)
    return h1, h2, h2 @ W3 + b3


def _softmax(z):
    z = z - z.max(axis=1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=1, keepdims=True)


def loss(params, X, ys, ym) -> float:
    _, _, o = forward(params, X)
    ps = _softmax(o[:, :S_CLASSES])
    pm = _softmax(o[:, S_CLASSES:])
    B = X.shape[0]
    ls = -np.log(ps[np.arange(B), ys])
    lm = -np.log(pm[np.arange(B), np.asarray(ym) - M_MIN])
    return float(np.mean(ls + lm))


def grads(params, X, ys, ym) -> np.ndarray:
    (W1, b1), (W2, b2), (W3, b3) = unpack(np.asarray(params, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    h1, h2, o = forward(params, X)
    B = X.shape[0]
    dO = np.concatenate([_softmax(o[:, :S_CLASSES]), _softmax(o[:, S_CLASSES:])], axis=1)
    dO[np.arange(B), ys] -= 1.0
    dO[np.arange(B), S_CLASSES + np.asarray(ym) - M_MIN] -= 1.0
    dO /= B
    dW3, db3 = h2.T @ dO, dO.sum(0)
    dh2 = (dO @ W3.T) * (h2 > 0)
    dW2, db2 = h1.T @ dh2, dh2.sum(0)
    dh1 = (dh2 @ W2.T) * (h1 > 0)
    dW1, db1 = X.T @ dh1, dh1.sum(0)
    return np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])


def predict(params, X):
    _, _, o = forward(params, X)
    return np.argmax(o[:, :S_CLASSES], axis=1), np.argmax(o[:, S_CLASSES:], axis=1) + M_MIN
