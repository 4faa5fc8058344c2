"""Pins of the oracle's QDWHpartial-EIG / -SVD against constructed spectra,
brute-force Jacobi, LAPACK and the paper's Theorem 1 and Section 7.4 numbers."""

import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from conftest import golden
from paper_2104_14186_gb300 import inputs as I

G = golden("paper_values.txt")

# Acceptance tolerances on the plain FP64 path.
LAM_TOL = 1e-12      # |lambda - lambda*| / ||A||_2
ORTH_TOL = 5e-15     # ||V^T V - I||_F / n
RES_TOL = 1e-13      # ||A V - V Lambda||_F / ||A||_F (SVD: ||A V - U S||_F / ||A||_F)
RES_TOL_T = 1e-13    # SVD transposed residual ||A^T U - V S||_F / ||A||_F (subspace containment)


def test_jacobi_bruteforce_against_constructed_spectrum():
    rng = np.random.default_rng(11)
    n = 40
    lam = np.sort(rng.uniform(-1, 1, n))
    Q = I.haar_orthogonal(n, rng)
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    l, V = O.jacobi_eig(A)
    assert np.max(np.abs(l - lam)) <= 1e-14
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= 1e-13
    assert np.linalg.norm(A @ V - V * l) <= 1e-13


def test_lanczos_bounds_known_spectrum():
    p = I.eig_uniform(400, 5)
    lo, rlo, hi, rhi = O.lanczos_extremes(lambda x: p.A @ x, 400, 30, 1)
    assert abs(lo - p.lam.min()) <= rlo + 1e-12
    assert abs(hi - p.lam.max()) <= rhi + 1e-12
    assert abs(lo - p.lam.min()) < 0.05 and abs(hi - p.lam.max()) < 0.05


@pytest.mark.parametrize("side", ["largest", "smallest"])
def test_threshold_interlacing(side):
    p = I.eig_uniform(300, 21, 0.1, side)
    eps_side = -1.0 if side == "largest" else 1.0
    lam_p = np.sort(eps_side * p.lam)
    for k in (1, 7, 30, 100):
        t = O.threshold_from_count_eig(p.A, eps_side, k, lam_p[-1] + 0.1, 16, 2, 3)
        assert np.count_nonzero(lam_p <= t + 1e-13) >= k
    q = I.svd_logspaced(200, 150, 4)
    for k in (1, 10, 60):
        sh = O.threshold_from_count_svd(q.A, k, 16, 2, 3)
        assert sh <= q.sigma[k - 1] * (1 + 1e-12)


@pytest.mark.parametrize("side,frac", [("largest", 0.10), ("smallest", 0.10), ("largest", 0.02), ("smallest", 0.3)])
def test_eig_constructed_spectrum_n512(side, frac):
    p = I.eig_uniform(512, 1000 + int(frac * 100), frac, side)
    r = O.qdwhp_eig(p.A, O.EigOptions(k=p.k, side=side))
    true = np.sort(p.lam)[::-1][: p.k] if side == "largest" else np.sort(p.lam)[: p.k]
    m = O.eig_metrics(p.A, r.lam, r.V, true)
    assert r.lam.shape == (p.k,) and r.V.shape == (512, p.k)
    assert m["lam_err"] <= LAM_TOL
    assert m["orth"] <= ORTH_TOL * 512
    assert m["resid"] <= RES_TOL
    assert r.ell >= p.k


def test_eig_against_bruteforce_jacobi():
    rng = np.random.default_rng(17)
    n = 48
    lam = rng.uniform(-1, 1, n)
    A = I.symmetric_with_spectrum(lam, rng)
    lj, Vj = O.jacobi_eig(A)
    for side, k in (("largest", 6), ("smallest", 10)):
        r = O.qdwhp_eig(A, O.EigOptions(k=k, side=side))
        ref = lj[::-1][:k] if side == "largest" else lj[:k]
        Vr = Vj[:, ::-1][:, :k] if side == "largest" else Vj[:, :k]
        assert np.max(np.abs(r.lam - ref)) <= 1e-13
        # same invariant subspace: by the Davis-Kahan sin-theta theorem each computed subspace is
        # within sqrt(2) ||A V - V Lambda||_F / gap (projector distance) of the exact one, the gap
        # being between the k-th and (k+1)-th eigenvalue
        srt = lj[::-1] if side == "largest" else lj
        gap = abs(srt[k - 1] - srt[k])
        res_q = np.linalg.norm(A @ r.V - r.V * r.lam)
        res_j = np.linalg.norm(A @ Vr - Vr * srt[:k])
        bound = np.sqrt(2.0) * (res_q + res_j) / gap
        assert np.linalg.norm(r.V @ r.V.T - Vr @ Vr.T) <= bound + 1e-14
        assert res_q <= 1e-13 * np.linalg.norm(A)


def test_eig_against_lapack_subset():
    p = I.eig_uniform(300, 77, 0.15, "largest")
    r = O.qdwhp_eig(p.A, O.EigOptions(k=p.k))
    ref = sla.eigh(p.A, eigvals_only=True, subset_by_index=[300 - p.k, 299])[::-1]
    assert np.max(np.abs(r.lam - ref)) <= 1e-13


def test_eig_paper_form_negative_eigenvalues():
    """Algorithm 1 as printed: negative eigenpairs given mu <= lambda_min."""
    rng = np.random.default_rng(5)
    n = 200
    lam = np.concatenate([rng.uniform(-1.0, -0.05, 25), rng.uniform(0.05, 1.0, 175)])
    A = I.symmetric_with_spectrum(lam, rng)
    l, V, info = O.qdwhp_eig_negative(A, mu=-1.05)
    assert np.max(np.abs(np.sort(l) - np.sort(lam[lam < 0]))) <= 1e-13
    assert np.linalg.norm(A @ V - V * l) <= 1e-13 * np.linalg.norm(A)


def test_theorem1_containment_bound():
    """Theorem 1: sin angle(V0, Q2) <= ||V0^T B||_2 / sigma_min(R11)."""
    rng = np.random.default_rng(9)
    n = 160
    lam = np.concatenate([rng.uniform(-1.0, -0.1, 20), rng.uniform(0.0, 1.0, 140)])
    Q = I.haar_orthogonal(n, rng)
    A = 0.5 * ((Q * lam) @ Q.T + ((Q * lam) @ Q.T).T)
    _, _, info = O.qdwhp_eig_negative(A, mu=-1.02)
    B, Qf, R, ind = info["B"], info["Q"], info["R"], info["ind"]
    V0 = Q[:, lam < 0]
    Q1 = Qf[:, :ind]
    sin_angle = np.linalg.norm(V0.T @ Q1, 2)
    bound = np.linalg.norm(V0.T @ B, 2) / np.linalg.svd(R[:ind, :ind], compute_uv=False).min()
    assert sin_angle <= bound * (1 + 1e-8) + 1e-15
    assert sin_angle <= 1e-12      # and it is tiny: Q2 contains V0 to working accuracy


def test_svd_constructed_spectrum():
    q = I.svd_logspaced(700, 500, 2000, 0.05)
    r = O.qdwhp_svd(q.A, O.SvdOptions(k=q.k))
    m = O.svd_metrics(q.A, r.sigma, r.U, r.V, q.sigma[: q.k])
    assert m["sigma_err"] <= LAM_TOL
    assert m["orthU"] <= ORTH_TOL * 500 and m["orthV"] <= ORTH_TOL * 500
    assert m["residV"] <= RES_TOL and m["residU"] <= RES_TOL_T


def test_svd_wide_matrix_is_solved_transposed():
    q = I.svd_logspaced(300, 240, 31, 0.1)
    At = np.asfortranarray(q.A.T)           # 240 x 300
    r = O.qdwhp_svd(At, O.SvdOptions(k=q.k))
    assert r.U.shape == (240, q.k) and r.V.shape == (300, q.k)
    m = O.svd_metrics(At, r.sigma, r.U, r.V, q.sigma[: q.k])
    assert m["sigma_err"] <= LAM_TOL and m["residV"] <= RES_TOL and m["residU"] <= RES_TOL_T


def test_svd_against_lapack():
    rng = np.random.default_rng(8)
    A = rng.standard_normal((260, 200))
    r = O.qdwhp_svd(A, O.SvdOptions(k=12))
    ref = np.linalg.svd(A, compute_uv=False)[:12]
    assert np.max(np.abs(r.sigma - ref)) <= 1e-12 * ref[0]


@pytest.mark.parametrize("s,key", [(0.1, "svd_geom_s_0.1_percent"), (0.01, "svd_geom_s_0.01_percent"),
                                   (1e-3, "svd_geom_s_1e-3_percent"), (1e-4, "svd_geom_s_1e-4_percent")])
def test_svd_threshold_fraction_paper_spectrum(s, key):
    """Section 7.4: for D[i] = 0.5^(100 i/N), s = 0.1, 0.01, 1e-3, 1e-4 select 3, 7, 10, 13 %
    of the triplets; small s takes the QR-based first step (Section 4.2)."""
    n = 300
    q = I.svd_geometric_half(n, 44)
    sig, U, V, info = O.qdwhp_svd_threshold(q.A, s, alpha=1.0)
    pct = 100.0 * sig.shape[0] / n
    assert abs(pct - float(G[key])) <= 1.0
    assert sig.shape[0] == np.count_nonzero(q.sigma >= s)
    assert np.max(np.abs(sig - q.sigma[: sig.shape[0]])) <= 1e-13
    if s <= 1e-3:
        assert info["n_qr"] >= 1
    assert np.linalg.norm(q.A @ V - U * sig) <= 1e-13 * np.linalg.norm(q.A)


def test_index_rule():
    R = np.diag([3.0, 1.0, 0.5, 0.009, 0.5, 1e-16])
    assert O.index_from_diag(R, float(G["index_tol"])) == 3
    assert O.index_from_diag(np.eye(4), 0.01) == 4


def test_degenerate_spectra():
    """Algorithm 1 divides by |mu|, which is 0 when the spectrum is one point (n = 1, a
    multiple of the identity, the zero matrix): then every vector is an eigenvector and the
    solver returns unit vectors with their Rayleigh quotients.  The zero matrix's singular
    values are all 0 (Algorithm 2's alpha = 0)."""
    r = O.qdwhp_eig(np.array([[3.0]]), O.EigOptions(k=1))
    assert r.lam.tolist() == [3.0] and r.V.tolist() == [[1.0]]
    for c in (2.5, 0.0, -1e-3):
        r = O.qdwhp_eig(c * np.eye(20), O.EigOptions(k=5, side="smallest"))
        assert np.all(r.lam == c) and np.array_equal(r.V, np.eye(20)[:, :5])
    s = O.qdwhp_svd(np.zeros((10, 8)), O.SvdOptions(k=3))
    assert np.all(s.sigma == 0.0)
    assert np.linalg.norm(s.U.T @ s.U - np.eye(3)) == 0.0 and np.linalg.norm(s.V.T @ s.V - np.eye(3)) == 0.0
    # k above the numerical rank: zero singular values are below every relative threshold
    # (Algorithm 2 keeps sigma >= s alpha), so the solver reports the shortfall
    rng = np.random.default_rng(1)
    B = rng.standard_normal((40, 10)) @ rng.standard_normal((10, 30))
    with pytest.raises(RuntimeError):
        O.qdwhp_svd(B, O.SvdOptions(k=15))
