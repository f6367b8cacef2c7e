"""Exponential Runge-Kutta steps in float64 -- test infrastructure only.

Follows Eq. (RK) of Sec. 2: for u' + A u = f(u),
    U_i  = u + tau * sum_{j<i} a_ij(-tau A) (f(U_j) - A u),
    u+   = u + tau * sum_i   b_i(-tau A)  (f(U_i) - A u),
with the Butcher tableaus of Table RK (exponential Euler; two stages with c2; three stages with
c2 and c3 = 2/3), each tableau entry a linear combination of phi_k(-c_j tau A).  Every entry is
applied as its own phi-action (no regrouping), with the phi-actions supplied by the caller
(``phi(t, v, p)`` -> array of phi_0..phi_p(-t A) v, e.g. ``phi.phi_dense`` or the spectral
oracles), and A u by the Kronecker-sum definition (Eq. (6)).

Pinned in tests/test_oracle_erk.py: f = 0 and f = const reproduce the exact solution
e^{-tau A} u + tau phi_1(-tau A) f for every method (the b_i sum to phi_1); against a stiff ODE
solver at tight tolerance the observed orders are 1, 2 and 3.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Tableau:
    name: str
    c: list            # nodes c_1..c_s
    a: dict            # (i, j) -> [(coef, k, c)] meaning coef * phi_k(-c tau A), 0-based i > j
    b: dict            # i -> [(coef, k, c)]


def euler() -> Tableau:
    return Tableau("euler", [0.0], {}, {0: [(1.0, 1, 1.0)]})


def rk2(c2: float = 0.5) -> Tableau:
    return Tableau("rk2", [0.0, c2],
                   {(1, 0): [(c2, 1, c2)]},
                   {0: [(1.0 - 1.0 / (2.0 * c2), 1, 1.0)], 1: [(1.0 / (2.0 * c2), 1, 1.0)]})


def rk3(c2: float = 1.0 / 3.0) -> Tableau:
    c3 = 2.0 / 3.0
    return Tableau("rk3", [0.0, c2, c3],
                   {(1, 0): [(c2, 1, c2)],
                    (2, 0): [(2.0 / 3.0, 1, c3), (-4.0 / (9.0 * c2), 2, c3)],
                    (2, 1): [(4.0 / (9.0 * c2), 2, c3)]},
                   {0: [(1.0, 1, 1.0), (-1.5, 2, 1.0)], 1: [], 2: [(1.5, 2, 1.0)]})


TABLEAUS = {"euler": euler, "rk2": rk2, "rk3": rk3}


def kron_sum_apply(factors, u: np.ndarray) -> np.ndarray:
    """A u for A = A^1 (+) ... (+) A^d (Eq. (6)): the sum of the mode-d products of u with A^d,
    u in C order with axis 0 the slowest."""
    shape = tuple(a.shape[0] for a in factors)
    U = np.asarray(u, dtype=np.float64).reshape(shape)
    out = np.zeros_like(U)
    for d, a in enumerate(factors):
        out += np.moveaxis(np.tensordot(a, U, axes=([1], [d])), 0, d)
    return out.ravel()


def allen_cahn(u: np.ndarray) -> np.ndarray:
    return u - u ** 3


def step(tab: Tableau, u: np.ndarray, tau: float, f, A_apply, phi) -> np.ndarray:
    u = np.asarray(u, dtype=np.float64)
    Au = A_apply(u)
    D = []
    for i in range(len(tab.c)):
        Ui = u.copy()
        for j in range(i):
            for coef, k, c in tab.a.get((i, j), []):
                Ui = Ui + tau * coef * phi(c * tau, D[j], k)[k]
        D.append(f(Ui) - Au)
    out = u.copy()
    for i in range(len(tab.c)):
        for coef, k, c in tab.b.get(i, []):
            out = out + tau * coef * phi(c * tau, D[i], k)[k]
    return out


def integrate(tab: Tableau, u0: np.ndarray, tau: float, nsteps: int, f, A_apply, phi) -> np.ndarray:
    u = np.asarray(u0, dtype=np.float64).copy()
    for _ in range(nsteps):
        u = step(tab, u, tau, f, A_apply, phi)
    return u
