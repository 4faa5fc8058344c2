"""Full symmetric eigendecomposition: QDWH-EIG (Section 3.2), plain FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

QDWH-EIG reaches, up to rounding, a result with a plain definition: every eigenpair
of the symmetric matrix.  `syev` is that definition (the LAPACK symmetric eigensolver
is its one step).  `qdwh_eig` follows the method of Section 3.2 step by step, as a
second, structural oracle: write A - sigma I = U_p H (eq. pdeig), so that
C = (I + U_p) / 2 = V_+ V_+^T projects onto the eigenvectors with eigenvalues above
sigma; take orthonormal bases of range(C) and of its complement, project A on each
(Rayleigh-Ritz) and recurse.  Readings (the paper does not fix them): the split point is
the mean eigenvalue trace(A) / n, the polar decomposition starts from ell_0 = 1e-15
(QR-based steps while c_k > 100), rank(C) = round(trace(C)), the bases come from
Householder QR with column pivoting of C, and problems of order <= `leaf` go to the
dense eigensolver.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .qdwh import qdwh_polar

ELL0_SPLIT = 1e-15


def syev(A: np.ndarray):
    """All eigenpairs of the symmetric A (the average of A and A^T), ascending."""
    S = 0.5 * (A + A.T)
    lam, V = np.linalg.eigh(S)
    return lam, V


def split(A: np.ndarray, sigma: float, alpha: float):
    """One spectral split (Section 3.2): U_p of (A - sigma I) / alpha, C = (I + U_p) / 2,
    r = round(trace C), [V1 V2] orthonormal with range(V1) = range(C).  Returns (r, V1, V2, C)."""
    n = A.shape[0]
    B = A - sigma * np.eye(n)
    Up, _, _ = qdwh_polar(B, alpha, ELL0_SPLIT)
    Up = 0.5 * (Up + Up.T)
    C = 0.5 * (np.eye(n) + Up)
    r = int(np.rint(np.trace(C)))
    r = min(max(r, 0), n)
    Q, _, _ = sla.qr(C, pivoting=True)
    return r, Q[:, :r], Q[:, r:], C


def qdwh_eig(A: np.ndarray, lo: float, hi: float, leaf: int = 64):
    """All eigenpairs of symmetric A with spectrum in [lo, hi] by recursive spectral
    splitting (Section 3.2).  Returns (lam, V), unordered."""
    A = 0.5 * (A + A.T)
    n = A.shape[0]
    if n <= leaf or hi - lo <= 1e-14 * max(abs(lo), abs(hi), 1e-300):
        return np.linalg.eigh(A)
    sigma = min(max(np.trace(A) / n, lo), hi)
    alpha = max(sigma - lo, hi - sigma)
    r, V1, V2, _ = split(A, sigma, alpha)
    if r in (0, n):
        return np.linalg.eigh(A)
    l1, W1 = qdwh_eig(V1.T @ A @ V1, sigma, hi, leaf)
    l2, W2 = qdwh_eig(V2.T @ A @ V2, lo, sigma, leaf)
    return np.concatenate([l1, l2]), np.hstack([V1 @ W1, V2 @ W2])
