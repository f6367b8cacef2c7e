"""Plain definitions of phi_l(M) v, M = -tau*(A^x (+) A^y (+) A^z).  Test infrastructure only.

phi_0(M) = e^M and phi_p(M) = int_0^1 e^{(1-theta)M} theta^{p-1}/(p-1)! dtheta for p >= 1
(Sec. 2.1, Eq. (3)).  Four independent evaluations:

O1 ``phi_dense``    -- assemble M densely and exponentiate the block matrix
                      [[M, v e_1^T], [0, J_p]] (J_p the p x p upper shift).  Its top-right
                      block column j is int_0^1 e^{(1-s)M} v s^{j-1}/(j-1)! ds = phi_j(M) v,
                      i.e. Eq. (3) applied to v.  scipy.linalg.expm is the library step.
O2 ``phi_spectral`` -- for symmetric factors diagonalised by the orthonormal sine (DST-I)
                      or Fourier transform: phi_l of the eigenvalue sums, entrywise.
O3 ``phi_sparse``   -- the same block matrix kept sparse; scipy.sparse.linalg.expm_multiply
                      computes its action on [v; 0] and on the unit vectors e_{N+j-1}.
O4 ``phi_mpmath``   -- O1 at 50 significant digits with mpmath (tiny sizes only).

Kronecker ordering (Sec. 2.2, Eq. (6)): for factors [A^1, ..., A^d] the first factor
acts on the slowest axis of the C-order vector, A = sum_d I (x) .. A^d .. (x) I.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg
import scipy.sparse
import scipy.sparse.linalg
import scipy.fft


# ----------------------------------------------------------------------------- scalar phi

def phi_scalar(l: int, z):
    """phi_l(z) for real or complex z (array-valued), float64/complex128.

    |z| <= 1 + l: Taylor series phi_l(z) = sum_k z^k/(k+l)! (from Eq. (3) by expanding
    e^{(1-theta)z}).  Otherwise the recurrence of Eq. (4) read backwards for scalars,
    phi_j(z) = (phi_{j-1}(z) - 1/(j-1)!)/z starting from phi_0 = e^z; for |z| > l each
    step divides the rounding error by |z|/j > 1, so it does not amplify it.
    Pinned in tests against mpmath quadrature of Eq. (3) and the closed forms of phi_1, phi_2.
    """
    z = np.asarray(z)
    cplx = np.iscomplexobj(z)
    z = z.astype(np.complex128 if cplx else np.float64)
    out = np.empty_like(z)
    small = np.abs(z) <= 1.0 + l
    if np.any(small):
        zs = z[small]
        acc = np.zeros_like(zs)
        # Horner over sum_{k=0}^{K} z^k/(k+l)!, K = 60 terms (|z|<=l+1 => tail < 1e-30 relative)
        K = 60 + 2 * l
        for k in range(K, -1, -1):
            acc = acc * zs + 1.0 / math.factorial(k + l)
        out[small] = acc
    big = ~small
    if np.any(big):
        zb = z[big]
        ph = np.exp(zb)
        for j in range(1, l + 1):
            ph = (ph - 1.0 / math.factorial(j - 1)) / zb
        out[big] = ph
    return out


# ----------------------------------------------------------------------------- assembly

def kron_sum_dense(factors) -> np.ndarray:
    """A = A^1 (+) ... (+) A^d as a dense matrix, Eq. (6) ordering (first factor slowest)."""
    sizes = [a.shape[0] for a in factors]
    N = int(np.prod(sizes))
    A = np.zeros((N, N))
    for d, a in enumerate(factors):
        left = int(np.prod(sizes[:d])) if d > 0 else 1
        right = int(np.prod(sizes[d + 1:])) if d + 1 < len(sizes) else 1
        A += np.kron(np.kron(np.eye(left), a), np.eye(right))
    return A


def kron_sum_sparse(factors) -> scipy.sparse.csr_matrix:
    sizes = [a.shape[0] for a in factors]
    N = int(np.prod(sizes))
    A = scipy.sparse.csr_matrix((N, N))
    for d, a in enumerate(factors):
        left = int(np.prod(sizes[:d])) if d > 0 else 1
        right = int(np.prod(sizes[d + 1:])) if d + 1 < len(sizes) else 1
        A = A + scipy.sparse.kron(scipy.sparse.kron(scipy.sparse.identity(left), scipy.sparse.csr_matrix(a)),
                                  scipy.sparse.identity(right), format="csr")
    return A.tocsr()


def _augmented_dense(M: np.ndarray, v: np.ndarray, p: int) -> np.ndarray:
    N = M.shape[0]
    Ahat = np.zeros((N + p, N + p))
    Ahat[:N, :N] = M
    Ahat[:N, N] = v
    for j in range(p - 1):
        Ahat[N + j, N + j + 1] = 1.0
    return Ahat


# ----------------------------------------------------------------------------- O1

def phi_dense(factors, tau: float, v: np.ndarray, p: int) -> np.ndarray:
    """O1: rows l = 0..p of phi_l(-tau*A) v from one dense expm of the augmented matrix."""
    M = -tau * kron_sum_dense(factors)
    N = M.shape[0]
    v = np.asarray(v, dtype=np.float64).ravel()
    out = np.empty((p + 1, N))
    if p == 0:
        out[0] = scipy.linalg.expm(M) @ v
        return out
    E = scipy.linalg.expm(_augmented_dense(M, v, p))
    out[0] = E[:N, :N] @ v
    for j in range(1, p + 1):
        out[j] = E[:N, N + j - 1]
    return out


def phi_dense_matrix(M: np.ndarray, v: np.ndarray, p: int) -> np.ndarray:
    """O1 for an already assembled matrix M (used by the identity checks)."""
    N = M.shape[0]
    out = np.empty((p + 1, N))
    if p == 0:
        out[0] = scipy.linalg.expm(M) @ v
        return out
    E = scipy.linalg.expm(_augmented_dense(M, v, p))
    out[0] = E[:N, :N] @ v
    for j in range(1, p + 1):
        out[j] = E[:N, N + j - 1]
    return out


# ----------------------------------------------------------------------------- O3

def phi_sparse(factors, tau: float, v: np.ndarray, p: int, orders=None) -> np.ndarray:
    """O3: phi_l(-tau*A) v via expm_multiply on the sparse augmented matrix.

    ``orders`` selects a subset of l in 0..p (default: all); rows come back in that order.
    """
    orders = list(range(p + 1)) if orders is None else list(orders)
    M = (-tau) * kron_sum_sparse(factors)
    N = M.shape[0]
    v = np.asarray(v, dtype=np.float64).ravel()
    if p == 0:
        return scipy.sparse.linalg.expm_multiply(M, v)[None, :]
    rows, cols, vals = [], [], []
    Mc = M.tocoo()
    rows += list(Mc.row); cols += list(Mc.col); vals += list(Mc.data)
    rows += list(range(N)); cols += [N] * N; vals += list(v)
    for j in range(p - 1):
        rows.append(N + j); cols.append(N + j + 1); vals.append(1.0)
    Ahat = scipy.sparse.csr_matrix((vals, (rows, cols)), shape=(N + p, N + p))
    B = np.zeros((N + p, len(orders)))
    for c, l in enumerate(orders):
        if l == 0:
            B[:N, c] = v
        else:
            B[N + l - 1, c] = 1.0
    X = scipy.sparse.linalg.expm_multiply(Ahat, B)
    return np.ascontiguousarray(X[:N, :].T)


# ----------------------------------------------------------------------------- O2

def dirichlet_eigs(n: int, coeff: float = 1.0, reaction: float = 0.0) -> np.ndarray:
    """Eigenvalues of coeff*(-D2) + reaction*I (Dirichlet, h = 1/(n+1)) in DST-I order."""
    k = np.arange(1, n + 1)
    h = 1.0 / (n + 1)
    return coeff * (2.0 - 2.0 * np.cos(k * np.pi / (n + 1))) / (h * h) + reaction


def phi_spectral_dirichlet(shape, coeffs, tau: float, v: np.ndarray, p: int, reactions=None) -> np.ndarray:
    """O2 for A^d = coeffs[d]*(-D2_dirichlet) + reactions[d]*I: the orthonormal DST-I
    diagonalises every factor, so phi_l(-tau*A) = Q phi_l(-tau*Lambda) Q^T entrywise."""
    reactions = reactions if reactions is not None else [0.0] * len(shape)
    V = np.asarray(v, dtype=np.float64).reshape(shape)
    Vh = scipy.fft.dstn(V, type=1, norm="ortho")
    lam = np.zeros(shape)
    for d, n in enumerate(shape):
        e = dirichlet_eigs(n, coeffs[d], reactions[d])
        sh = [1] * len(shape)
        sh[d] = n
        lam = lam + e.reshape(sh)
    z = -tau * lam
    out = np.empty((p + 1, int(np.prod(shape))))
    for l in range(p + 1):
        out[l] = scipy.fft.idstn(phi_scalar(l, z) * Vh, type=1, norm="ortho").ravel()
    return out


def phi_spectral_periodic(shape, coeffs, tau: float, v: np.ndarray, p: int) -> np.ndarray:
    """O2 for A^d = coeffs[d]*(-D2_periodic) on [0,1): the DFT diagonalises it with
    eigenvalues coeff*(2 - 2cos(2 pi k/n))*n^2."""
    V = np.asarray(v, dtype=np.float64).reshape(shape)
    Vh = np.fft.fftn(V)
    lam = np.zeros(shape)
    for d, n in enumerate(shape):
        k = np.arange(n)
        e = coeffs[d] * (2.0 - 2.0 * np.cos(2.0 * np.pi * k / n)) * n * n
        sh = [1] * len(shape)
        sh[d] = n
        lam = lam + e.reshape(sh)
    z = -tau * lam
    out = np.empty((p + 1, int(np.prod(shape))))
    for l in range(p + 1):
        out[l] = np.real(np.fft.ifftn(phi_scalar(l, z) * Vh)).ravel()
    return out


# ----------------------------------------------------------------------------- O4

def phi_mpmath(factors, tau: float, v: np.ndarray, p: int, dps: int = 50) -> np.ndarray:
    """O4: O1's augmented matrix exponentiated in mpmath at ``dps`` digits (tiny N only)."""
    import mpmath as mp
    with mp.workdps(dps):
        A = kron_sum_dense(factors)
        N = A.shape[0]
        v = np.asarray(v, dtype=np.float64).ravel()
        size = N + max(p, 1)
        Ah = mp.zeros(size, size)
        t = mp.mpf(tau)
        for i in range(N):
            for j in range(N):
                if A[i, j] != 0.0:
                    Ah[i, j] = -t * mp.mpf(A[i, j])
        if p > 0:
            for i in range(N):
                Ah[i, N] = mp.mpf(v[i])
            for j in range(p - 1):
                Ah[N + j, N + j + 1] = 1
        E = mp.expm(Ah)
        out = np.empty((p + 1, N))
        for i in range(N):
            out[0, i] = float(mp.fsum(E[i, k] * mp.mpf(v[k]) for k in range(N)))
            for j in range(1, p + 1):
                out[j, i] = float(E[i, N + j - 1])
        return out


# ----------------------------------------------------------------------------- helpers

def apply_kron(mats, V: np.ndarray) -> np.ndarray:
    """(mats[0] (x) mats[1] (x) ...) vec(V) for a C-order tensor V (Eq. (8) as mode products)."""
    X = V
    for d, E in enumerate(mats):
        X = np.moveaxis(np.tensordot(E, X, axes=([1], [d])), 0, d)
    return X


def rel_err_2(approx: np.ndarray, exact: np.ndarray) -> float:
    """Relative 2-norm error ||approx - exact|| / ||exact||."""
    den = np.linalg.norm(exact)
    return float(np.linalg.norm(approx - exact) / (den if den > 0 else 1.0))
