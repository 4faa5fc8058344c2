"""QDWH iteration: dynamical weights and the two practical step forms (FP64).

Section 3.1 of the paper.  The iteration (eq. polar-itr) is
    X_{k+1} = X_k (a_k I + b_k X_k^T X_k)(I + c_k X_k^T X_k)^{-1},
whose scalar form is r_k(x) = x (a_k + b_k x^2) / (1 + c_k x^2); it is never
evaluated in that inverse form.  The two step forms used instead are the
QR-based update (eq. practical-polar-qr) and the Cholesky-based update
(eq. practical-polar-chol).
"""

from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

# Unit roundoff u = 2^-53.  Section 5's listing stops on |L - 1| >= 5 eps, with eps
# the spacing of doubles at 1 (2^-52 = 2u); the reading taken is 5 * 2^-52.
EPS = 2.0 ** -52
CONV_TOL = 5.0 * EPS


def dwh_weights(ell: float) -> tuple[float, float, float, float]:
    """Weights (a, b, c) of the (3,2) Zolotarev step for the interval [ell, 1]
    and the updated lower bound ell_next = r(ell).

    Section 3.1 (weights chosen so that r_k is the scaled Zolotarev function of
    type (3,2) on [-1,-ell] U [ell,1], ell_k = r_k(ell_{k-1})) and the weight
    lines of the Section 5 listing:
        L2 = ell^2,  d = cbrt(4 (1 - L2) / L2^2),
        a = sqrt(1 + d) + 0.5 sqrt(8 - 4 d + 8 (2 - L2) / (L2 sqrt(1 + d))),
        b = (a - 1)^2 / 4,  c = a + b - 1,  ell_next = ell (a + b L2) / (1 + c L2).
    For ell >= 1 the function is Halley's: a = 3, b = 1, c = 3.
    """
    if ell >= 1.0:
        return 3.0, 1.0, 3.0, 1.0
    L2 = ell * ell
    d = np.cbrt(4.0 * (1.0 - L2) / (L2 * L2))
    sqd = math.sqrt(1.0 + d)
    a = sqd + 0.5 * math.sqrt(8.0 - 4.0 * d + 8.0 * (2.0 - L2) / (L2 * sqd))
    b = (a - 1.0) ** 2 / 4.0
    c = a + b - 1.0
    ell_next = ell * (a + b * L2) / (1.0 + c * L2)
    return a, b, c, min(ell_next, 1.0)


def dwh_schedule(ell0: float, max_iter: int = 12, fixed_iters: int | None = None):
    """Weights of every iteration from ell0.

    With ``fixed_iters`` (QDWHpartial-EIG, Algorithm 1 step 2: three iterations
    for s = 0.2, two for s = 0.875) exactly that many steps; otherwise iterate
    while |ell - 1| >= 5 eps (Algorithm 2 step 2, Section 5 listing).
    Returns a list of (a, b, c, ell_before, ell_after).
    """
    out = []
    ell = ell0
    while True:
        if fixed_iters is not None:
            if len(out) >= fixed_iters:
                break
        elif abs(ell - 1.0) < CONV_TOL:
            break
        if len(out) >= max_iter:
            break
        a, b, c, nxt = dwh_weights(ell)
        out.append((a, b, c, ell, nxt))
        ell = nxt
    return out


def rational_map(x, a: float, b: float, c: float):
    """Scalar r(x) = x (a + b x^2) / (1 + c x^2) (Section 3.1)."""
    x = np.asarray(x, dtype=np.float64)
    return x * (a + b * x * x) / (1.0 + c * x * x)


def qdwh_chol_step(X: np.ndarray, a: float, b: float, c: float) -> np.ndarray:
    """Cholesky-based QDWH step, eq. practical-polar-chol:
        Z = I + c X^T X,  W = chol(Z) (upper, Z = W^T W),
        X_next = (b/c) X + (a - b/c) (X W^{-1}) W^{-T}.
    """
    n = X.shape[1]
    Z = np.eye(n) + c * (X.T @ X)
    W = sla.cholesky(Z, lower=False)
    # Y1 = X W^{-1}  <=>  W^T Y1^T = X^T
    Y1t = sla.solve_triangular(W, X.T, trans="T", lower=False)
    # Y2 = Y1 W^{-T} <=>  W Y2^T = Y1^T
    Y2t = sla.solve_triangular(W, Y1t, trans="N", lower=False)
    return (b / c) * X + (a - b / c) * Y2t.T


def qdwh_qr_step(X: np.ndarray, a: float, b: float, c: float) -> np.ndarray:
    """QR-based QDWH step, eq. practical-polar-qr:
        [sqrt(c) X; I] = [Q1; Q2] R,
        X_next = (b/c) X + (1/sqrt(c)) (a - b/c) Q1 Q2^T.
    """
    m, n = X.shape
    S = np.vstack([math.sqrt(c) * X, np.eye(n)])
    Q, _ = np.linalg.qr(S, mode="reduced")
    Q1, Q2 = Q[:m], Q[m:]
    return (b / c) * X + (a - b / c) / math.sqrt(c) * (Q1 @ Q2.T)


def qdwh_polar(A: np.ndarray, alpha: float, ell0: float, c_qr: float = 100.0, max_iter: int = 12):
    """Full QDWH polar decomposition A = U_p H (Section 3.1): X_0 = A / alpha,
    QR-based steps while c_k > c_qr, Cholesky-based afterwards, until ell reaches
    1 within 5 eps.  Returns (U_p, H, schedule)."""
    X = A / alpha
    sched = dwh_schedule(ell0, max_iter=max_iter)
    for a, b, c, _, _ in sched:
        X = qdwh_qr_step(X, a, b, c) if c > c_qr else qdwh_chol_step(X, a, b, c)
    H = X.T @ A
    H = 0.5 * (H + H.T)
    return X, H, sched
