"""Full spectra: QDWH-EIG and QDWH-SVD (Section 3.2), plain FP64.

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

QDWH-SVD reaches, up to rounding, every singular triplet of A; `gesvd` is that
definition (the LAPACK SVD as its one step).  `qdwh_svd` follows Section 3.2: the
polar decomposition A = U_p H by QDWH, the symmetric eigendecomposition H = V Sigma V^T
(here by `qdwh_eig`, the same spectral divide and conquer), and U = U_p V.  Readings
(the paper does not fix them): A with m < n is solved as A^T with U and V swapped;
alpha = ||A||_2; the polar decomposition starts from ell_0 = 1e-15, so its guarantee
covers sigma_min / sigma_max >= 1e-15; an eigenvalue lambda of H taken negative by
rounding gives sigma = |lambda| with the matching column of U negated (A v = lambda U_p v);
and when the smallest sigma is at most 1e-14 alpha (numerically rank-deficient A, whose
polar factor QDWH does not settle on the null directions), U is replaced by the
orthonormal factor of its Householder QR with the signs of diag(R), which leaves the
other columns unchanged to rounding and completes the null ones orthonormally.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .qdwh import qdwh_polar

ELL0_SPLIT = 1e-15
ELL0_SVD = 1e-15
ORTH_FIX_SVD = 1e-14


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


def gesvd(A: np.ndarray):
    """All singular triplets of A, thin (p = min(m, n)): (sigma descending, U m x p, V n x p)."""
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    return s, U, Vt.T


def qdwh_svd(A: np.ndarray, leaf: int = 64):
    """QDWH-SVD (Section 3.2): A = U_p H, H = V Sigma V^T, U = U_p V.  Returns
    (sigma descending, U, V, info) with info["orthonormalized"] set when U was completed
    by its QR (numerically rank-deficient A)."""
    m, n = A.shape
    if m < n:
        s, U, V, info = qdwh_svd(A.T, leaf)
        return s, V, U, info
    alpha = float(np.linalg.norm(A, 2))
    if alpha == 0.0:
        return np.zeros(n), np.eye(m, n), np.eye(n), {"orthonormalized": False, "zero": True}
    Up, H, sched = qdwh_polar(A, alpha, ELL0_SVD)
    lam, W = qdwh_eig(H, -0.01 * alpha, 1.01 * alpha, leaf)
    order = np.argsort(-np.abs(lam), kind="stable")
    lam, W = lam[order], W[:, order]
    sigma = np.abs(lam)
    sgn = np.where(lam < 0.0, -1.0, 1.0)
    U = (Up @ W) * sgn[None, :]
    fixed = bool(sigma[-1] <= ORTH_FIX_SVD * alpha)
    if fixed:
        Q, R = np.linalg.qr(U)
        d = np.where(np.diag(R) < 0.0, -1.0, 1.0)
        U = Q * d[None, :]
    return sigma, U, W, {"orthonormalized": fixed, "zero": False, "polar_steps": len(sched)}
