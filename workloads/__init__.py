"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module builds the *problem data* only: the 1D finite-difference factors A^d of a
Kronecker-sum operator A = A^x (+) A^y (+) A^z, the input vectors v and the per-config
parameter sets.  It holds none of the method's arithmetic (no exponentials, no
quadrature, no phi-functions), so the CUDA path and the oracle can both consume it
without sharing any computation.

Sign convention (Sec. 2.1, Eq. (1) and Sec. 4.1): the library computes phi_l(-tau*A) v
for a matrix A that is positive (semi)definite "like minus a Laplacian".  The factors
built here are therefore A^d = -c*D2 (+ advection), i.e. the dissipative operator with
the minus sign already applied.

Layout: a 3D vector is C-order [n_x][n_y][n_z] (z fastest); A^x acts on the slowest
axis, as in the Kronecker ordering of Eq. (6)/(8).  Matrices are dense, row-major,
float64 numpy arrays.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


# ----------------------------------------------------------------------------- 1D factors

def d2_dirichlet(n: int, length: float = 1.0) -> np.ndarray:
    """Second-order central difference on n interior points of [0, length], Dirichlet.

    h = length/(n+1); D2 = tridiag(1, -2, 1)/h^2.  (Negative semidefinite.)
    """
    h = length / (n + 1)
    D = np.zeros((n, n))
    idx = np.arange(n)
    D[idx, idx] = -2.0
    D[idx[:-1], idx[:-1] + 1] = 1.0
    D[idx[1:], idx[1:] - 1] = 1.0
    return D / (h * h)


def d1_upwind_dirichlet(n: int, length: float = 1.0) -> np.ndarray:
    """First-order backward (upwind for positive velocity) difference (u_i - u_{i-1})/h."""
    h = length / (n + 1)
    D = np.zeros((n, n))
    idx = np.arange(n)
    D[idx, idx] = 1.0
    D[idx[1:], idx[1:] - 1] = -1.0
    return D / h


def d2_periodic(n: int, length: float = 1.0) -> np.ndarray:
    """Central difference on the periodic grid x_i = i*h, h = length/n."""
    h = length / n
    D = np.zeros((n, n))
    idx = np.arange(n)
    D[idx, idx] = -2.0
    D[idx, (idx + 1) % n] += 1.0
    D[idx, (idx - 1) % n] += 1.0
    return D / (h * h)


def laplacian_factor(n: int, coeff: float = 1.0, reaction: float = 0.0) -> np.ndarray:
    """A^d = -coeff*D2 + reaction*I on n interior Dirichlet points of [0,1] (SPD)."""
    return -coeff * d2_dirichlet(n) + reaction * np.eye(n)


def convdiff_factor(n: int, diffusion: float = 0.01, velocity: float = 1.0) -> np.ndarray:
    """A^d = -diffusion*D2 + velocity*D1_upwind on [0,1], Dirichlet (nonsymmetric)."""
    return -diffusion * d2_dirichlet(n) + velocity * d1_upwind_dirichlet(n)


def periodic_diffusion_factor(n: int, coeff: float) -> np.ndarray:
    """A^d = -coeff*D2_periodic on [0,1) (symmetric positive semidefinite)."""
    return -coeff * d2_periodic(n)


# ----------------------------------------------------------------------------- vectors

def uniform_vector(shape, seed: int, low: float = -1.0, high: float = 1.0) -> np.ndarray:
    """v ~ U(low, high) from numpy's default_rng(seed), float64, C-order, flattened."""
    rng = np.random.default_rng(seed)
    return rng.uniform(low, high, size=int(np.prod(shape)))


def sine_vector(shape) -> np.ndarray:
    """b = prod_d sin(pi x_d) at the interior nodes x = i/(n_d+1) (the Sec. 4.1 initial datum)."""
    grids = [np.sin(np.pi * np.arange(1, n + 1) / (n + 1)) for n in shape]
    out = grids[0]
    for g in grids[1:]:
        out = np.multiply.outer(out, g)
    return np.ascontiguousarray(out).ravel()


# ----------------------------------------------------------------------------- configs

@dataclass
class Problem:
    """One phi-action problem: factors A^d, step tau, orders 0..l_max, tolerance."""
    name: str
    factors: list            # list of (n_d x n_d) float64 arrays, slowest axis first
    tau: float
    l_max: int
    tol: float
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def shape(self):
        return tuple(a.shape[0] for a in self.factors)

    @property
    def N(self) -> int:
        return int(np.prod(self.shape))

    def vector(self) -> np.ndarray:
        return uniform_vector(self.shape, self.seed)


def laplace2d(n: int = 32, tau: float = 1e-3, l_max: int = 3, tol: float = 1e-10,
              seed: int = 0) -> Problem:
    """2D Dirichlet Laplacian, A = A^x (+) A^y with A^d = -D2 on n interior points."""
    a = laplacian_factor(n)
    return Problem(f"laplace2d_n{n}", [a, a.copy()], tau, l_max, tol, seed)


def convdiff3d(n: int = 128, tau: float = 1e-2, l_max: int = 3, tol: float = 1e-10,
               seed: int = 0, shape=None) -> Problem:
    """3D convection-diffusion, A^d = -0.01*D2 + 1.0*D1_upwind (nonsymmetric)."""
    shape = shape or (n, n, n)
    facs = [convdiff_factor(k) for k in shape]
    name = "convdiff3d_" + "x".join(str(k) for k in shape)
    return Problem(name, facs, tau, l_max, tol, seed)


BATCH_SIZES = (64, 96, 128, 192, 256)


def batched_uneven3d(count: int = 32, seed: int = 3, sizes=BATCH_SIZES, nrhs: int = 4):
    """Instances of 3D diffusion with uneven sizes, coefficient c ~ U(0.1,1), tau ~ logU(1e-4,1e-1).

    Returns a list of dicts {shape, coeff, tau, rhs_seeds}.  The factors are
    A^d = -c*D2 on n_d interior Dirichlet points.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        shape = tuple(int(s) for s in rng.choice(sizes, size=3))
        coeff = float(rng.uniform(0.1, 1.0))
        tau = float(10.0 ** rng.uniform(-4.0, -1.0))
        out.append(dict(shape=shape, coeff=coeff, tau=tau,
                        rhs_seeds=[100 + nrhs * i + r for r in range(nrhs)]))
    return out


def batched_instance_factors(inst) -> list:
    return [laplacian_factor(n, inst["coeff"]) for n in inst["shape"]]


def allen_cahn2d(n: int = 2048, eps: float = 0.01, seed: int = 4):
    """Periodic [0,1)^2 Allen-Cahn u' = eps^2*Lap(u) + u - u^3; returns (factor, u0)."""
    a = periodic_diffusion_factor(n, eps * eps)
    rng = np.random.default_rng(seed)
    u0 = rng.uniform(-0.05, 0.05, size=n * n)
    return a, u0


def log_uniform(rng, lo: float, hi: float, size=None):
    return 10.0 ** rng.uniform(math.log10(lo), math.log10(hi), size=size)
