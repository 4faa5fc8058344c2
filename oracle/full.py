"""Full spectra: QDWH-EIG and QDWH-SVD (Section 3.2), plain FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

QDWH-EIG reaches, up to rounding, a result with a plain definition: every eigenpair
of the symmetric matrix.  `syev` is that definition (the LAPACK symmetric eigensolver
is its one step).  `qdwh_eig` follows the method of Section 3.2 step by step, as a
second, structural oracle: write A - sigma I = U_p H (eq. pdeig), so that
C = (I + U_p) / 2 = V_+ V_+^T projects onto the eigenvectors with eigenvalues above
sigma; take orthonormal bases of range(C) and of its complement, project A on each
(Rayleigh-Ritz) and recurse.  Readings (the paper does not fix them): the split point is
an estimate of the median eigenvalue from the Gauss quadrature of 30 Lanczos steps on A
(`quadrature_median`, a midpoint between two distinct nodes), then the mean eigenvalue
trace(A) / n and the middle of [lo, hi], the first whose split is two-sided, resolved
(trace(C) - ||C||_F^2 <= 0.05, C being a projector to rounding) and exact to rounding
(||V2^T A V1||_F <= 64 eps sqrt(n) alpha); the polar decomposition starts from
ell_0 = 1e-15
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

from scipy.linalg import eigh_tridiagonal

from .partial import lanczos_tridiagonal
from .qdwh import qdwh_polar

ELL0_SPLIT = 1e-15
ELL0_SVD = 1e-15
ORTH_FIX_SVD = 1e-14
UNRESOLVED = 0.05
OFFBLOCK = 64 * 2.0 ** -52
SLQ_STEPS = 30
SLQ_SEED = 4242


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


def quadrature_nodes_weights(alpha: np.ndarray, beta: np.ndarray):
    """Gauss quadrature of the Lanczos tridiagonal (Golub-Welsch): nodes = eigenvalues of T
    (ascending), weights = squared first components of its eigenvectors."""
    m = alpha.shape[0]
    if m == 1:
        return alpha.copy(), np.ones(1)
    theta, S = eigh_tridiagonal(alpha, beta[: m - 1])
    return theta, S[0] ** 2


def quadrature_median(A: np.ndarray, seed: int = SLQ_SEED):
    """Split point near the median eigenvalue of symmetric A, or None.  With the quadrature
    nodes ascending and c_j the cumulative (normalised) weights, j* is the first node with
    c_j >= 1/2.  Nodes converge onto clusters, so the candidates are the midpoints beside
    theta_j*: of theta_{j*-1} and theta_j* (predicting a fraction c_{j*-1} at or below it)
    and of theta_j* and theta_{j*+1} (predicting c_j*).  The candidate whose prediction lies
    strictly inside (0, 1) and nearest 1/2 is returned."""
    n = A.shape[0]
    alpha, beta = lanczos_tridiagonal(lambda x: A @ x, n, SLQ_STEPS, seed)
    theta, w = quadrature_nodes_weights(alpha, beta)
    m = theta.shape[0]
    c = np.cumsum(w / np.sum(w))
    j = int(min(np.searchsorted(c, 0.5), m - 1))
    # two nodes may sit on one cluster: a midpoint is taken only between distinct nodes
    sep = 1e-8 * max(theta[-1] - theta[0], np.max(np.abs(theta)), 1e-300)
    cands = []
    a = j - 1
    while a >= 0 and theta[j] - theta[a] <= sep:
        a -= 1
    if a >= 0:
        cands.append((0.5 * (theta[a] + theta[j]), c[a]))
    b = j + 1
    while b < m and theta[b] - theta[j] <= sep:
        b += 1
    if b < m:
        cands.append((0.5 * (theta[j] + theta[b]), c[b - 1]))
    cands = [x for x in cands if 1e-12 < x[1] < 1.0 - 1e-12]
    if not cands:
        return None
    return float(min(cands, key=lambda x: abs(x[1] - 0.5))[0])


def qdwh_eig(A: np.ndarray, lo: float, hi: float, leaf: int = 64):
    """All eigenpairs of symmetric A with spectrum in [lo, hi] by recursive spectral
    splitting (Section 3.2).  Returns (lam, V), unordered."""
    A = 0.5 * (A + A.T)
    n = A.shape[0]
    if n <= leaf or hi - lo <= 1e-14 * max(abs(lo), abs(hi), 1e-300):
        return np.linalg.eigh(A)
    med = quadrature_median(A)
    cands = ([med] if med is not None else []) + [np.trace(A) / n, 0.5 * (lo + hi)]
    for cand in cands:
        sigma = min(max(cand, lo), hi)
        alpha = max(sigma - lo, hi - sigma)
        r, V1, V2, C = split(A, sigma, alpha)
        if not (0 < r < n and np.trace(C) - np.sum(C * C) <= UNRESOLVED):
            continue
        # the split's backward error, at the level of the rounding of the products
        if np.linalg.norm(V2.T @ A @ V1) <= OFFBLOCK * np.sqrt(n) * alpha:
            break
    else:
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
