"""Zolo-PD: the polar decomposition by Zolotarev's best rational approximation of the
sign function (FP64).  TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 3.1 presents QDWH as the type (3, 2) member of the Zolotarev family and names the
higher-order variant (Zolo-PD) as the path to fewer iterations; the conclusion lists it
as future work.  This module writes that variant out from its definition (Nakatsukasa and
Freund, SIAM Review 58 (2016)):

* On [ell, 1] the best type (2r+1, 2r) rational approximation of sign(x), scaled to take
  the value 1 at x = 1, is
      Z(x) = M x prod_{j=1..r} (x^2 + c_{2j}) / (x^2 + c_{2j-1}),
      c_i = ell^2 sn^2(i K' / (2r+1); ell') / cn^2(i K' / (2r+1); ell'),
  with ell' = sqrt(1 - ell^2), K' = K(ell') and M = prod_j (1 + c_{2j-1}) / (1 + c_{2j}).
  It maps [ell, 1] onto [Z(ell), 1]; r = 1 is the QDWH function of Section 3.1.
* Partial fractions: Z(x) = M x (1 + sum_j a_j / (x^2 + c_{2j-1})),
      a_j = -prod_k (c_{2j-1} - c_{2k}) / prod_{k != j} (c_{2j-1} - c_{2k-1}).
* One iteration on the matrix X: X <- M (X + sum_j a_j X (X^T X + c_{2j-1} I)^{-1}), the r
  terms independent of one another.  A term is formed with a Cholesky factorisation of
  X^T X + c I, or, when that matrix may be ill conditioned (1 / c_{2j-1} > c_qr, the bound
  QDWH applies to its own Cholesky step), from the QR factorisation
  [X; sqrt(c) I] = [Q1; Q2] R as Q1 Q2^T / sqrt(c).
* ell_{k+1} = Z(ell_k); iterate until |ell - 1| < 5 eps, as for QDWH.

The elliptic functions are scipy's (parameter m = ell'^2); K' uses ellipkm1(ell^2) so that
it stays accurate for small ell.  ellipj loses accuracy as m -> 1: from ell = 1e-3 up the
map is exact to rounding for r <= 8 (the coefficients to ~3e-11 relative at 1e-3), while at
some smaller ell (1e-5, 1e-4) it is off by up to 1e-8.  The oracle is meant for ell >= 1e-3,
the range of the partial solvers' thresholds on the test problems that compare against it.
"""

from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla
from scipy.special import ellipj, ellipkm1

from .qdwh import CONV_TOL


def zolo_coeffs(ell: float, r: int):
    """(c_1..c_2r, a_1..a_r, M) of the type (2r+1, 2r) Zolotarev function on [ell, 1]."""
    if not (0.0 < ell < 1.0) or r < 1:
        raise ValueError("need 0 < ell < 1 and r >= 1")
    Kp = float(ellipkm1(ell * ell))          # K(m) at m = 1 - ell^2
    u = np.arange(1, 2 * r + 1) * Kp / (2 * r + 1)
    sn, cn, _, _ = ellipj(u, 1.0 - ell * ell)
    c = ell * ell * (sn / cn) ** 2
    codd, ceven = c[0::2], c[1::2]
    a = np.empty(r)
    for j in range(r):
        num = np.prod(codd[j] - ceven)
        den = np.prod([codd[j] - codd[k] for k in range(r) if k != j])
        a[j] = -num / den
    M = float(np.prod((1.0 + codd) / (1.0 + ceven)))
    return c, a, M


def zolo_map(x, c: np.ndarray, M: float):
    """Scalar Z(x) = M x prod_j (x^2 + c_{2j}) / (x^2 + c_{2j-1})."""
    x = np.asarray(x, dtype=np.float64)
    out = M * x
    for j in range(c.shape[0] // 2):
        out = out * (x * x + c[2 * j + 1]) / (x * x + c[2 * j])
    return out


def zolo_schedule(ell0: float, r: int, max_iter: int = 12):
    """[(c, a, M, ell, ell_next), ...] from ell0 until |ell - 1| < 5 eps."""
    out = []
    ell = float(ell0)
    while abs(ell - 1.0) >= CONV_TOL and len(out) < max_iter:
        c, a, M = zolo_coeffs(ell, r)
        nxt = min(float(zolo_map(ell, c, M)), 1.0)
        out.append((c, a, M, ell, nxt))
        ell = nxt
    return out


def zolo_term_chol(X: np.ndarray, G: np.ndarray, cj: float) -> np.ndarray:
    """X (G + cj I)^{-1} with G = X^T X, by Cholesky: G + cj I = W^T W."""
    n = X.shape[1]
    W = sla.cholesky(G + cj * np.eye(n), lower=False)
    Y1t = sla.solve_triangular(W, X.T, trans="T", lower=False)     # (X W^{-1})^T
    Y2t = sla.solve_triangular(W, Y1t, trans="N", lower=False)     # (X W^{-1} W^{-T})^T
    return Y2t.T


def zolo_term_qr(X: np.ndarray, cj: float) -> np.ndarray:
    """X (X^T X + cj I)^{-1} from [X; sqrt(cj) I] = [Q1; Q2] R: Q1 Q2^T / sqrt(cj)."""
    m, n = X.shape
    Q, _ = np.linalg.qr(np.vstack([X, math.sqrt(cj) * np.eye(n)]), mode="reduced")
    return (Q[:m] @ Q[m:].T) / math.sqrt(cj)


def zolo_step(X: np.ndarray, c: np.ndarray, a: np.ndarray, M: float, c_qr: float = 100.0):
    """One Zolo-PD iteration; returns (X_next, number of QR-formed terms)."""
    G = X.T @ X
    acc = X.copy()
    n_qr = 0
    for j in range(a.shape[0]):
        cj = float(c[2 * j])
        if 1.0 / cj > c_qr:
            T = zolo_term_qr(X, cj)
            n_qr += 1
        else:
            T = zolo_term_chol(X, G, cj)
        acc += a[j] * T
    return M * acc, n_qr


def zolo_polar(A: np.ndarray, alpha: float, ell0: float, r: int, c_qr: float = 100.0):
    """Zolo-PD polar decomposition A = U_p H from X_0 = A / alpha (sigma(X_0) in
    [ell0, 1]).  Returns (U_p, H, schedule)."""
    X = A / alpha
    sched = zolo_schedule(ell0, r)
    for c, a, M, _, _ in sched:
        X, _ = zolo_step(X, c, a, M, c_qr)
    H = X.T @ A
    H = 0.5 * (H + H.T)
    return X, H, sched
