"""Pins of the full-spectrum oracle (QDWH-EIG, Section 3.2) against constructed spectra,
the brute-force Jacobi eigensolver and the projector identity after eq. pdeig."""

import numpy as np

import oracle as O
from paper_2104_14186_gb300 import inputs as I


def test_syev_constructed_and_bruteforce():
    rng = np.random.default_rng(31)
    lam = np.sort(rng.uniform(-2, 1, 90))
    A = I.symmetric_with_spectrum(lam, rng)
    l, V = O.syev(A)
    assert np.max(np.abs(l - lam)) <= 1e-14 * 2
    assert np.linalg.norm(V.T @ V - np.eye(90)) <= 1e-13
    assert np.linalg.norm(A @ V - V * l) <= 1e-13 * np.linalg.norm(A)
    B = I.symmetric_with_spectrum(lam[:40], rng)
    lj, _ = O.jacobi_eig(B)
    assert np.max(np.abs(O.syev(B)[0] - np.sort(lj))) <= 1e-14 * 2


def test_split_projector_identity():
    """(I + U_p)/2 = V+ V+^T: its trace counts the eigenvalues above sigma and its range is
    their invariant subspace (a dropped 1/2, a sign flip of U_p or a wrong shift fails)."""
    rng = np.random.default_rng(5)
    n = 120
    lam = np.concatenate([rng.uniform(-1.0, -0.05, 50), rng.uniform(0.1, 1.0, 70)])
    Q = I.haar_orthogonal(n, rng)
    A = 0.5 * ((Q * lam) @ Q.T + ((Q * lam) @ Q.T).T)
    sigma = 0.02
    r, V1, V2, C = O.full.split(A, sigma, 1.05)
    assert r == np.count_nonzero(lam > sigma) == 70
    Vp = Q[:, lam > sigma]
    assert np.linalg.norm(C - Vp @ Vp.T) <= 1e-13
    # the bases split A: the off-diagonal block vanishes
    assert np.linalg.norm(V2.T @ A @ V1) <= 1e-13
    assert np.linalg.norm(np.hstack([V1, V2]).T @ np.hstack([V1, V2]) - np.eye(n)) <= 1e-13


def test_qdwh_eig_recursion_constructed():
    rng = np.random.default_rng(12)
    n = 200
    lam = np.concatenate([rng.uniform(-1, 1, 150), np.full(30, 0.25), 0.5 + 1e-9 * rng.standard_normal(20)])
    A = I.symmetric_with_spectrum(lam, rng)
    l, V = O.full.qdwh_eig(A, -1.1, 1.1, leaf=24)
    order = np.argsort(l)
    l, V = l[order], V[:, order]
    assert np.max(np.abs(l - np.sort(lam))) <= 1e-13
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= 5e-15 * n
    assert np.linalg.norm(A @ V - V * l) <= 1e-13 * np.linalg.norm(A)


def svd_check(A, s, U, V, s_true, tol_s=1e-13):
    m, n = A.shape
    p = min(m, n)
    assert s.shape == (p,) and U.shape == (m, p) and V.shape == (n, p)
    assert np.all(np.diff(s) <= 0)
    assert np.max(np.abs(s - s_true)) <= tol_s * max(np.max(s_true), 1e-300)
    mt = O.svd_metrics(A, s, U, V)
    assert mt["orthU"] <= 5e-15 * p and mt["orthV"] <= 5e-15 * p, mt
    assert mt["residV"] <= 1e-13 and mt["residU"] <= 1e-13, mt


def test_gesvd_definition_constructed():
    """The definition against a constructed spectrum and against the eigenvalues of A^T A
    from the symmetric eigensolver (a different LAPACK path)."""
    rng = np.random.default_rng(41)
    sig = np.sort(rng.uniform(0.1, 3.0, 60))[::-1]
    A = I.general_with_singular_values(90, sig, rng)
    s, U, V = O.full.gesvd(A)
    svd_check(A, s, U, V, sig)
    ev = np.sort(np.linalg.eigvalsh(A.T @ A))[::-1]
    assert np.max(np.abs(s ** 2 - ev)) <= 1e-13 * 9.0
    # brute force: one-sided Jacobi eigenvalues of A^T A on a small case
    B = A[:30, :20]
    lj, _ = O.jacobi_eig(B.T @ B)
    assert np.max(np.abs(np.sort(O.full.gesvd(B)[0] ** 2) - np.sort(lj))) <= 1e-13 * np.max(lj)


def test_qdwh_svd_graded_tall_and_wide():
    """sigma log-spaced over 12 decades (inside ell_0 = 1e-15): every triplet meets the FP64
    tolerances, for m > n and, through the transpose, m < n (swapped U, V fail the shapes or
    the residuals)."""
    p = I.svd_logspaced(150, 100, 7)
    s, U, V, info = O.full.qdwh_svd(p.A, leaf=24)
    assert not info["orthonormalized"]
    svd_check(p.A, s, U, V, p.sigma)
    s2, U2, V2, _ = O.full.qdwh_svd(np.asfortranarray(p.A.T), leaf=24)
    svd_check(np.asfortranarray(p.A.T), s2, U2, V2, p.sigma)


def test_qdwh_svd_matches_definition_square():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((120, 120))
    s, U, V, _ = O.full.qdwh_svd(A, leaf=30)
    s0, U0, V0 = O.full.gesvd(A)
    svd_check(A, s, U, V, s0)
    # singular vectors agree with the definition's up to sign (random A: simple spectrum)
    dots = np.abs(np.sum(U * U0, axis=0))
    gaps = np.minimum(np.r_[np.inf, -np.diff(s0)], np.r_[-np.diff(s0), np.inf])
    ok = gaps > 1e-6 * s0[0]
    assert np.all(np.abs(dots[ok] - 1.0) <= 1e-8)


def test_qdwh_svd_rank_deficient_and_zero():
    """20 exact zero singular values: U is completed orthonormally (QR with the signs of
    diag R); the zero matrix returns sigma = 0 and unit vectors."""
    rng = np.random.default_rng(9)
    sig = np.concatenate([np.sort(rng.uniform(0.5, 2.0, 80))[::-1], np.zeros(20)])
    A = I.general_with_singular_values(140, sig, rng)
    s, U, V, info = O.full.qdwh_svd(A, leaf=32)
    assert info["orthonormalized"]
    svd_check(A, s, U, V, sig)
    s, U, V, info = O.full.qdwh_svd(np.zeros((30, 20)))
    assert np.all(s == 0.0) and info["zero"]
    assert np.array_equal(U, np.eye(30, 20)) and np.array_equal(V, np.eye(20))


def test_quadrature_exact_to_degree_2m_minus_1():
    """Gauss quadrature from m Lanczos steps integrates polynomials of degree <= 2m - 1
    exactly against the spectral measure of the start vector: sum_j w_j theta_j^p =
    q0^T A^p q0 (Golub-Welsch; a wrong weight vector or node set fails this)."""
    from oracle.partial import STREAM_LANCZOS, lanczos_tridiagonal
    from oracle.rng import uniform_pm1
    rng = np.random.default_rng(2)
    n, m, seed = 60, 6, 99
    A = I.symmetric_with_spectrum(rng.uniform(-1.0, 2.0, n), rng)
    al, be = lanczos_tridiagonal(lambda x: A @ x, n, m, seed)
    theta, w = O.full.quadrature_nodes_weights(al, be)
    q0 = uniform_pm1(seed ^ STREAM_LANCZOS, n)
    q0 = q0 / np.linalg.norm(q0)
    v = q0.copy()
    for p in range(2 * m):
        mom = q0 @ v
        assert abs(np.sum(w * theta ** p) - mom) <= 1e-12 * max(1.0, np.sum(np.abs(w * theta ** p))), p
        v = A @ v


def test_quadrature_median_balances_graded_spectra():
    """Sigma log-spaced over 12 decades: the mean splits 88/12, the quadrature estimate
    far nearer the middle; a two-point spectrum gets a point strictly between its values."""
    rng = np.random.default_rng(3)
    lam = 10.0 ** (-12.0 * np.arange(1024) / 1023)
    A = I.symmetric_with_spectrum(lam, rng)
    s = O.full.quadrature_median(A)
    assert np.mean(lam <= np.mean(lam)) > 0.85
    assert 0.2 <= np.mean(lam <= s) <= 0.8
    lam2 = np.concatenate([np.zeros(20), np.ones(180)])
    s2 = O.full.quadrature_median(I.symmetric_with_spectrum(lam2, rng))
    assert 0.0 < s2 < 1.0


def test_unresolved_split_is_detected():
    """A split point on a 30-fold eigenvalue: those directions sit within rounding (~1e-16)
    of sigma, below the polar resolution ell_0 = 1e-15, so C has eigenvalues strictly inside
    (0, 1) there and trace(C) - ||C||_F^2 = sum p (1 - p) is far above the 0.05 acceptance
    bound (at most 30/4); a split point in a gap gives ~0."""
    rng = np.random.default_rng(5)
    lam = np.concatenate([rng.uniform(-1.0, -0.1, 50), np.full(30, 0.25), rng.uniform(0.5, 1.0, 40)])
    A = I.symmetric_with_spectrum(lam, rng)
    _, _, _, C = O.full.split(A, 0.25, 1.3)
    assert 1.0 <= np.trace(C) - np.sum(C * C) <= 7.5 + 1e-9
    _, _, _, C = O.full.split(A, 0.4, 1.45)
    assert abs(np.trace(C) - np.sum(C * C)) <= 1e-10
