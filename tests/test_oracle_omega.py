"""Pins of the oracle's Gaussian Omega option of the extraction QR (Section 4.1: the QR of
(r(A~) + I) Omega is rank revealing with high probability, so diag(R) tracks the singular
values of R11 and the index rule with tol = 0.01 is safe) and of its Box-Muller generator."""

import math

import numpy as np
import pytest
import scipy.stats

import oracle as O
from paper_2104_14186_gb300 import inputs as I


def test_gaussian_is_standard_normal():
    """Kolmogorov-Smirnov against N(0, 1), the first four moments, and no correlation between
    the cos and sin halves of a Box-Muller pair (a dropped factor 2 in the radius, a wrong
    sign of the log or a shared angle fails one of these)."""
    g = O.gaussian(12345, 200_001)
    assert g.shape == (200_001,) and np.all(np.isfinite(g))
    assert scipy.stats.kstest(g, "norm").pvalue > 1e-3
    assert abs(g.mean()) < 0.01 and abs(g.var() - 1.0) < 0.01
    assert abs(scipy.stats.skew(g)) < 0.03 and abs(scipy.stats.kurtosis(g)) < 0.06
    a, b = g[0:200_000:2], g[1:200_000:2]
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.01
    # a prefix of a longer draw is the shorter draw (counter-based: output i depends on i only)
    assert np.array_equal(O.gaussian(12345, 7), g[:7])


def test_omega_unit_scale():
    """Entries N(0, 1/n): column norms near 1 and the largest singular value near the
    Marchenko-Pastur edge 2 of a square Gaussian matrix, so B Omega keeps B's scale."""
    n = 400
    Om = O.gaussian_omega(n, 99)
    assert Om.shape == (n, n)
    cn = np.linalg.norm(Om, axis=0)
    assert abs(cn.mean() - 1.0) < 0.02
    s = np.linalg.svd(Om, compute_uv=False)
    assert 1.85 < s[0] < 2.15 and s[-1] > 0.0


def _kahan(n: int, c: float) -> np.ndarray:
    s = math.sqrt(1.0 - c * c)
    K = np.triu(-c * np.ones((n, n)), 1) + np.eye(n)
    return np.diag(s ** np.arange(n)) @ K


def test_kahan_matrix_needs_omega():
    """Kahan's matrix (n = 100, c = 0.2) is upper triangular with every |diagonal| >= 0.13, yet
    its smallest singular value is ~4e-9.  The unpivoted QR is the matrix itself, so the index
    rule finds no small diagonal and captures nothing (ell = 0).  With Omega the QR reveals
    the rank: ell >= 1, the null direction lies in Q2 within Theorem 1's bound, and the
    smallest diagonal of R11 is within a factor 100 of sigma_min(R11)."""
    K = _kahan(100, 0.2)
    U, S, _ = np.linalg.svd(K)
    assert S[-1] < 1e-8 and np.abs(np.diag(K)).min() > 0.13
    v0 = U[:, -1:]
    for tol in (0.1, 0.01):
        _, _, R, ind = O.extraction_qr(K, tol)
        assert ind == K.shape[0]
        F, Qf, R, ind = O.extraction_qr(K, tol, omega_seed=7)
        assert ind < K.shape[0]
        smin = np.linalg.svd(R[:ind, :ind], compute_uv=False).min()
        sin_angle = np.linalg.norm(v0.T @ Qf[:, :ind], 2)
        bound = np.linalg.norm(v0.T @ F, 2) / smin
        assert sin_angle <= bound * (1 + 1e-8) + 1e-15
        assert sin_angle <= 1e-5
        assert np.abs(np.diag(R)[:ind]).min() <= 100.0 * smin


def test_theorem1_bound_with_omega():
    """Theorem 1 for B Omega: sin angle(V0, Q2) <= ||V0^T B Omega||_2 / sigma_min(R11), and Q2
    contains the negative eigenvectors to working accuracy at the printed tol = 0.01."""
    rng = np.random.default_rng(9)
    n = 160
    lam = np.concatenate([rng.uniform(-1.0, -0.1, 20), rng.uniform(0.0, 1.0, 140)])
    Q = I.haar_orthogonal(n, rng)
    A = 0.5 * ((Q * lam) @ Q.T + ((Q * lam) @ Q.T).T)
    neg, V, info = O.qdwhp_eig_negative(A, mu=-1.02, omega_seed=5)
    F, Qf, R, ind = info["F"], info["Q"], info["R"], info["ind"]
    assert not np.array_equal(F, info["B"])
    V0 = Q[:, lam < 0]
    sin_angle = np.linalg.norm(V0.T @ Qf[:, :ind], 2)
    bound = np.linalg.norm(V0.T @ F, 2) / np.linalg.svd(R[:ind, :ind], compute_uv=False).min()
    assert sin_angle <= bound * (1 + 1e-8) + 1e-15
    assert sin_angle <= 1e-12
    assert np.max(np.abs(np.sort(neg) - np.sort(lam[lam < 0]))) <= 1e-13


def test_tol_001_with_omega_meets_the_tolerance_where_unpivoted_does_not():
    """n = 300, 5 % smallest, seed 5013: at the printed tol = 0.01 the unpivoted QR's residual
    is 3.3e-13 (diag(R) overestimates sigma_min(R11)); with Omega it is below 1e-13, and the
    eigenvalues match the constructed spectrum either way."""
    p = I.eig_uniform(300, 5013, 0.05, side="smallest")
    want = np.sort(p.lam)[: p.k]
    r0 = O.qdwhp_eig(p.A, O.EigOptions(k=p.k, side="smallest", tol=0.01))
    r1 = O.qdwhp_eig(p.A, O.EigOptions(k=p.k, side="smallest", tol=0.01, use_omega=True))
    m0 = O.eig_metrics(p.A, r0.lam, r0.V, want)
    m1 = O.eig_metrics(p.A, r1.lam, r1.V, want)
    assert m0["resid"] > 1e-13
    assert m1["resid"] <= 1e-13 and m1["lam_err"] <= 1e-12 and m1["orth"] <= 5e-15 * 300


@pytest.mark.parametrize("seed", [5001, 5006, 5011])
def test_eig_and_svd_with_omega_at_tol_001(seed):
    """Both partial solvers with (tol = 0.01, Omega) on constructed spectra at the FP64
    tolerances."""
    p = I.eig_uniform(200, seed, 0.2, side="largest")
    r = O.qdwhp_eig(p.A, O.EigOptions(k=p.k, tol=0.01, use_omega=True))
    m = O.eig_metrics(p.A, r.lam, r.V, np.sort(p.lam)[::-1][: p.k])
    assert m["lam_err"] <= 1e-12 and m["orth"] <= 5e-15 * 200 and m["resid"] <= 1e-13, m
    q = I.svd_logspaced(300, 200, seed, 0.05)
    r = O.qdwhp_svd(q.A, O.SvdOptions(k=q.k, tol=0.01, use_omega=True))
    m = O.svd_metrics(q.A, r.sigma, r.U, r.V, q.sigma[: q.k])
    assert m["sigma_err"] <= 1e-12 and m["residV"] <= 1e-13 and m["residU"] <= 1e-13, m
