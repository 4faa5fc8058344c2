"""Brute-force cyclic Jacobi eigensolver for small symmetric matrices (n <= 64).

An independent check of the oracle's partial results: the classical two-sided
Jacobi method (Jacobi 1846; rotation formulas as in Golub and Van Loan,
Matrix Computations, 4th ed., Section 8.5), written with plain Python loops
over the (p, q) pairs.  It uses no LAPACK routine.
"""

import math

import numpy as np


def jacobi_eig(A: np.ndarray, max_sweeps: int = 60):
    """All eigenpairs of symmetric A, eigenvalues ascending.  Returns (lam, V)."""
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    V = np.eye(n)
    for _ in range(max_sweeps):
        off = math.sqrt(np.sum(np.triu(A, 1) ** 2))
        if off <= 1e-18 * math.sqrt(np.sum(A * A)):
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                if apq == 0.0:
                    continue
                # t = tan(theta) is the smaller root of t^2 + 2 tau t - 1 = 0
                tau = (A[q, q] - A[p, p]) / (2.0 * apq)
                t = math.copysign(1.0, tau) / (abs(tau) + math.sqrt(1.0 + tau * tau))
                c = 1.0 / math.sqrt(1.0 + t * t)
                s = t * c
                # A <- J^T A J with J the rotation in the (p, q) plane
                ap = A[:, p].copy()
                aq = A[:, q].copy()
                A[:, p] = c * ap - s * aq
                A[:, q] = s * ap + c * aq
                ap = A[p, :].copy()
                aq = A[q, :].copy()
                A[p, :] = c * ap - s * aq
                A[q, :] = s * ap + c * aq
                A[p, q] = A[q, p] = 0.0
                vp = V[:, p].copy()
                vq = V[:, q].copy()
                V[:, p] = c * vp - s * vq
                V[:, q] = s * vp + c * vq
    lam = np.diag(A).copy()
    order = np.argsort(lam, kind="stable")
    return lam[order], V[:, order]
