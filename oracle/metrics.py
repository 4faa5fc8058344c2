"""Accuracy metrics (Section 7.3, eqs. orth, sv, allsv) plus the normwise forms
used as acceptance tolerances:

  eigenvalue error     max_i |lambda_i - lambda*_i| / ||A||_2
  orthogonality        ||V^T V - I||_F            (and the paper's ||I - V^T V||_F / n)
  residual             ||A V - V Lambda||_F / ||A||_F
  per-column residual  max_i ||A v_i - lambda_i v_i||_2  (eq. allsv)
  relative error       ||Lambda - Delta||_F / ||Delta||_F  (eq. sv)

For an n x k matrix V the paper's ||I - V V^T||_F / n is read as the k x k
form ||I - V^T V||_F / n (the n x n form is at least sqrt(n - k)).
"""

import numpy as np


def eig_metrics(A: np.ndarray, lam: np.ndarray, V: np.ndarray, lam_true: np.ndarray | None = None) -> dict:
    n, k = V.shape
    norm2 = np.linalg.norm(A, 2) if n <= 2048 else None
    normF = np.linalg.norm(A, "fro")
    R = A @ V - V * lam[None, :]
    out = {
        "orth": float(np.linalg.norm(V.T @ V - np.eye(k), "fro")),
        "resid": float(np.linalg.norm(R, "fro") / normF),
        "resid_col_max": float(np.max(np.linalg.norm(R, axis=0))) if k else 0.0,
    }
    out["orth_paper"] = out["orth"] / n
    if lam_true is not None:
        scale = norm2 if norm2 is not None else float(np.max(np.abs(lam_true)))
        out["lam_err"] = float(np.max(np.abs(lam - lam_true)) / scale) if k else 0.0
        out["lam_relF"] = float(np.linalg.norm(lam - lam_true) / max(np.linalg.norm(lam_true), 1e-300))
    return out


def svd_metrics(A: np.ndarray, sigma: np.ndarray, U: np.ndarray, V: np.ndarray,
                sigma_true: np.ndarray | None = None) -> dict:
    m, n = A.shape
    k = sigma.shape[0]
    normF = np.linalg.norm(A, "fro")
    RV = A @ V - U * sigma[None, :]
    RU = A.T @ U - V * sigma[None, :]
    out = {
        "orthU": float(np.linalg.norm(U.T @ U - np.eye(k), "fro")),
        "orthV": float(np.linalg.norm(V.T @ V - np.eye(k), "fro")),
        "residV": float(np.linalg.norm(RV, "fro") / normF),
        "residU": float(np.linalg.norm(RU, "fro") / normF),
        "resid_col_max": float(max(np.max(np.linalg.norm(RV, axis=0)), np.max(np.linalg.norm(RU, axis=0)))) if k else 0.0,
    }
    if sigma_true is not None:
        scale = float(np.max(sigma_true))
        out["sigma_err"] = float(np.max(np.abs(sigma - sigma_true)) / scale) if k else 0.0
        out["sigma_relF"] = float(np.linalg.norm(sigma - sigma_true) / max(np.linalg.norm(sigma_true), 1e-300))
    return out
