"""Algorithms 1, 2 and 6 (fixed and adaptive quadrature with scaling and modified squaring),
restated step by step in float64 with library matrix exponentials.  Test infrastructure only.

These follow the paper's order and notation and serve two purposes: (i) pin the
reading of the paper against the plain definition (``phi.phi_dense``), and (ii) give
the exact intermediate quantities (scaled-level y_j, squaring steps) against which the
GPU path's stages can be compared.  Mode products use ``phi.apply_kron`` (tensordot).

Reading (listed in the design notes): Algorithm 6 returns phi_1..phi_p only; phi_0 is
added as (e^{M^x} (x) e^{M^y} (x) e^{M^z}) v by Eq. (7)-(8).  The squaring update of
Algorithm 6 is simultaneous: every y-hat_i is formed from the previous y_1..y_i.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

from . import planner
from .phi import apply_kron


def alg1_fixed(Ms, v: np.ndarray, p: int, x: np.ndarray, w: np.ndarray):
    """Algorithm 1 for the matrix M = (+)_d Ms[d]: returns y_j ~ phi_j(M) v, j = 1..p.

    v_i = (x)_d e^{(1-x_i) Ms[d]} v ;  y_j = sum_i w_i x_i^{j-1}/(j-1)! v_i.
    """
    shape = tuple(a.shape[0] for a in Ms)
    V = np.asarray(v, dtype=np.float64).reshape(shape)
    vs = []
    for xi in x:
        mats = [scipy.linalg.expm((1.0 - xi) * a) for a in Ms]
        vs.append(apply_kron(mats, V).ravel())
    ys = []
    for j in range(1, p + 1):
        y = np.zeros(V.size)
        for i in range(len(x)):
            y += w[i] * x[i] ** (j - 1) / math.factorial(j - 1) * vs[i]
        ys.append(y)
    return ys


def alg2_adaptive_cc(Ms, v: np.ndarray, p: int, tol: float, max_nodes: int = 385):
    """Algorithm 2 for M = (+)_d Ms[d]: nested Clenshaw-Curtis rules with 2n+1 points, n = 3,
    6, 12, ...; each refinement evaluates the integrand only at the new (odd-indexed) nodes and
    re-forms y_j with the new rule's weights, until err = max_j ||y_j - y~_j||_inf / ||y_j||_inf
    <= tol.  Returns (y_1..y_p, nodes used, final err).  Reading: a y_j that is zero with a
    zero change counts as converged; a rule above max_nodes stops with err > tol."""
    shape = tuple(a.shape[0] for a in Ms)
    V = np.asarray(v, dtype=np.float64).reshape(shape)

    def integrand(xi):
        return apply_kron([scipy.linalg.expm((1.0 - xi) * a) for a in Ms], V).ravel()

    def weighted(x, w, vs):
        ys = []
        for j in range(1, p + 1):
            y = np.zeros(V.size)
            for i in range(len(x)):
                y += w[i] * x[i] ** (j - 1) / math.factorial(j - 1) * vs[i]
            ys.append(y)
        return ys

    n = 3
    x, w = planner.clenshaw_curtis_01(2 * n)
    vs = [integrand(xi) for xi in x]
    y = weighted(x, w, vs)
    err = math.inf
    while err > tol:
        if 4 * n + 1 > max_nodes:
            break
        n = 2 * n
        ytil = y
        x, w = planner.clenshaw_curtis_01(2 * n)
        new = [None] * (2 * n + 1)
        for i in range(2 * n + 1):
            new[i] = vs[i // 2] if i % 2 == 0 else integrand(x[i])   # even points are the old rule's
        vs = new
        y = weighted(x, w, vs)
        err = 0.0
        for j in range(p):
            d = np.max(np.abs(y[j] - ytil[j]))
            m_ = np.max(np.abs(y[j]))
            err = max(err, d / m_ if m_ > 0 else (math.inf if d > 0 else 0.0))
    return y, len(x), err


def remark_combo(factors, tau: float, B, x: np.ndarray, w: np.ndarray) -> np.ndarray:
    """The Remark after Algorithm 2: sum_j phi_j(M) b_j ~ sum_i w_i e^{(1-x_i)M} sum_j
    x_i^{j-1}/(j-1)! b_j for M = -tau A (no scaling), B = [b_1, ..., b_p]."""
    Ms = [-tau * np.asarray(a, dtype=np.float64) for a in factors]
    shape = tuple(a.shape[0] for a in Ms)
    out = np.zeros(int(np.prod(shape)))
    for xi, wi in zip(x, w):
        z = np.zeros_like(out)
        for j in range(1, len(B) + 1):
            z += xi ** (j - 1) / math.factorial(j - 1) * np.asarray(B[j - 1], dtype=np.float64)
        mats = [scipy.linalg.expm((1.0 - xi) * a) for a in Ms]
        out += wi * apply_kron(mats, z.reshape(shape)).ravel()
    return out


def alg6_phiquadmv(factors, tau: float, v: np.ndarray, p: int, tol: float,
                   s: int | None = None, m: int | None = None, rule: str = planner.GAUSS,
                   return_stages: bool = False):
    """Algorithm 6 for M = -tau*A, phi_0..phi_p; returns array (p+1, N) [and stages].

    (s, m) default to Algorithm 5 with alpha = tau*sum ||A^d||_inf, beta = 1, eps = tol.
    """
    Ms = [-tau * np.asarray(a, dtype=np.float64) for a in factors]
    shape = tuple(a.shape[0] for a in Ms)
    V = np.asarray(v, dtype=np.float64).reshape(shape)
    out = np.empty((p + 1, V.size))
    out[0] = apply_kron([scipy.linalg.expm(a) for a in Ms], V).ravel()
    stages = {}
    if p == 0:
        return (out, stages) if return_stages else out
    if s is None or m is None:
        alpha = planner.alpha_inf(factors, tau)
        s_, m_, _ = planner.setup_quadrature(tol, p, alpha, 1.0, planner.CC if rule == "cc_adaptive" else rule)
        s = s_ if s is None else s
        m = m_ if m is None else m
    scaled = [a / 2.0 ** s for a in Ms]
    if rule == "cc_adaptive":
        y, used, err = alg2_adaptive_cc(scaled, V.ravel(), p, tol)
        stages["nodes"], stages["err"] = used, err
    else:
        if rule == planner.GAUSS:
            x, w = planner.gauss_legendre_01(m)
        else:
            x, w = planner.clenshaw_curtis_01(m - 1)
        y = alg1_fixed(scaled, V.ravel(), p, x, w)
    stages["scaled"] = [yy.copy() for yy in y]
    F = [scipy.linalg.expm(a) for a in scaled]          # e^{2^{-s} M^d}
    for k in range(s):
        Gy = [apply_kron(F, yi.reshape(shape)).ravel() for yi in y]
        yhat = []
        for i in range(1, p + 1):
            acc = Gy[i - 1].copy()
            for j in range(1, i + 1):
                acc += y[j - 1] / math.factorial(i - j)
            yhat.append(acc / 2.0 ** i)
        y = yhat
        stages[f"square{k}"] = [yy.copy() for yy in y]
        if k < s - 1:
            F = [f @ f for f in F]                        # e^{2^{k+1-s} M^d} = (e^{2^{k-s} M^d})^2
    for j in range(1, p + 1):
        out[j] = y[j - 1]
    stages["s"], stages["m"] = s, m
    return (out, stages) if return_stages else out
