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
