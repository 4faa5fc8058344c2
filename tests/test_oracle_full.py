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
