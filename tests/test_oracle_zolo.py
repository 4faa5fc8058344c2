"""Pins of the Zolo-PD oracle (the higher-order Zolotarev variant of QDWH, Section 3.1)
against facts that do not come from its own formulas: the QDWH weights (r = 1 is the
QDWH function), Chebyshev alternation of the best approximation, the composition law
of Zolotarev functions, the spectral-map identity of one matrix iteration in both the
Cholesky and QR forms, the polar factor from the SVD, and the partial solvers run with
Zolo-PD against constructed spectra."""

import numpy as np
import pytest

import oracle as O
from oracle import zolo as Z
from paper_2104_14186_gb300 import inputs as I


@pytest.mark.parametrize("ell", [0.9, 0.2, 1e-2, 1e-3])
def test_r1_is_the_qdwh_function(ell):
    """Type (3, 2): c_1 = 1 / c, c_2 = a / b, M = b / c with the dynamical weights of Section 3.1."""
    c, a_pf, M = Z.zolo_coeffs(ell, 1)
    a, b, cq, _ = O.dwh_weights(ell)
    assert abs(1.0 / c[0] - cq) <= 1e-12 * cq
    assert abs(c[1] - a / b) <= 1e-12 * (a / b)
    assert abs(M - b / cq) <= 1e-12 * (b / cq)
    x = np.linspace(ell, 1.0, 101)
    # the maps agree to the rounding of the coefficients amplified by c (1.6e4 at ell = 1e-3)
    assert np.max(np.abs(Z.zolo_map(x, c, M) - O.rational_map(x, a, b, cq))) <= 1e-12


@pytest.mark.parametrize("ell,r", [(0.2, 2), (0.25, 3), (1e-2, 4), (0.05, 5)])
def test_chebyshev_alternation(ell, r):
    """The scaled error 1 - Z(x) / m, m = (1 + Z(ell)) / 2, equioscillates: it takes its
    extreme magnitude E with alternating signs at 2r + 2 points of [ell, 1] (the
    characterisation of the best type (2r+1, 2r) approximation of 1 there)."""
    c, _, M = Z.zolo_coeffs(ell, r)
    x = np.geomspace(ell, 1.0, 400001)
    f = Z.zolo_map(x, c, M)
    assert abs(f[-1] - 1.0) <= 1e-14 and np.all(f <= 1.0 + 1e-13) and np.all(f >= f[0] - 1e-13)
    m = 0.5 * (1.0 + f[0])
    e = 1.0 - f / m
    E = np.max(np.abs(e))
    # local extrema of e (interior) plus both ends
    d = np.diff(e)
    idx = np.concatenate([[0], np.nonzero(np.sign(d[1:]) != np.sign(d[:-1]))[0] + 1, [x.size - 1]])
    ext = e[idx]
    assert np.all(np.abs(np.abs(ext) - E) <= 1e-6 * E + 1e-15)
    assert np.all(np.sign(ext[1:]) != np.sign(ext[:-1]))
    assert ext.size == 2 * r + 2


@pytest.mark.parametrize("ell,r", [(0.1, 1), (0.3, 2)])
def test_composition_law(ell, r):
    """Z_{2r+1}( Z_{2r+1}(x; ell); Z_{2r+1}(ell; ell) ) = Z_{(2r+1)^2}(x; ell) on [ell, 1]."""
    c1, _, M1 = Z.zolo_coeffs(ell, r)
    ell1 = float(Z.zolo_map(ell, c1, M1))
    c2, _, M2 = Z.zolo_coeffs(ell1, r)
    R = ((2 * r + 1) ** 2 - 1) // 2
    c3, _, M3 = Z.zolo_coeffs(ell, R)
    x = np.geomspace(ell, 1.0, 2001)
    two = Z.zolo_map(Z.zolo_map(x, c1, M1), c2, M2)
    one = Z.zolo_map(x, c3, M3)
    assert np.max(np.abs(two - one)) <= 1e-12


@pytest.mark.parametrize("c_qr", [100.0, 0.0])
def test_step_spectral_map(c_qr):
    """X = U diag(s) V^T -> U diag(Z(s)) V^T in one iteration; c_qr = 0 forces the QR form
    of every term, 100 lets the well-conditioned ones use Cholesky."""
    rng = np.random.default_rng(4)
    ell, r = 0.05, 3
    s = np.concatenate([[ell, 1.0], rng.uniform(ell, 1.0, 58)])
    U = I.haar_orthogonal(60, rng, 90)
    V = I.haar_orthogonal(60, rng)
    X = (U * s) @ V.T
    c, a, M = Z.zolo_coeffs(ell, r)
    Xn, n_qr = Z.zolo_step(X, c, a, M, c_qr)
    assert n_qr == (3 if c_qr == 0.0 else sum(1.0 / c[0::2] > 100.0))
    assert np.linalg.norm(Xn - (U * Z.zolo_map(s, c, M)) @ V.T) <= 1e-13 * np.sqrt(60)
    # partial fractions = product form
    y = np.linspace(ell, 1.0, 50)
    pf = M * y * (1.0 + sum(a[j] / (y * y + c[2 * j]) for j in range(r)))
    assert np.max(np.abs(pf - Z.zolo_map(y, c, M))) <= 1e-13


@pytest.mark.parametrize("ell0,r,iters", [(0.2, 2, 2), (0.2, 1, 3), (1e-3, 8, 2), (1e-3, 1, 4)])
def test_polar_factor_and_iteration_counts(ell0, r, iters):
    """Zolo-PD returns the polar factor U V^T; r = 1 takes QDWH's counts (3 from 0.2, 4 from
    1e-3), higher orders fewer."""
    rng = np.random.default_rng(8)
    n = 50
    s = np.geomspace(ell0, 1.0, n)
    U = I.haar_orthogonal(n, rng, 70)
    V = I.haar_orthogonal(n, rng)
    A = (U * s) @ V.T
    Up, H, sched = Z.zolo_polar(A, 1.0, ell0, r)
    assert len(sched) == iters
    assert abs(sched[-1][4] - 1.0) < 5 * 2.0 ** -52
    assert np.linalg.norm(Up - U @ V.T) <= 1e-13 * n
    assert np.linalg.norm(H - (V * s) @ V.T) <= 1e-13 * n


def test_partial_solvers_with_zolo():
    """QDWHpartial-EIG and -SVD with Zolo-PD (r = 2) in place of QDWH meet the FP64
    tolerances against the constructed spectra."""
    p = I.eig_uniform(256, 31, 0.10)
    r = O.qdwhp_eig(p.A, O.EigOptions(k=p.k, zolo_r=2))
    m = O.eig_metrics(p.A, r.lam, r.V, np.sort(p.lam)[::-1][: p.k])
    assert len(r.info["sched"]) == 2
    assert m["lam_err"] <= 1e-12 and m["orth"] <= 5e-15 * 256 and m["resid"] <= 1e-13, m
    q = I.svd_logspaced(300, 200, 5, 0.05)
    rs = O.qdwhp_svd(q.A, O.SvdOptions(k=q.k, zolo_r=2))
    mt = O.svd_metrics(q.A, rs.sigma, rs.U, rs.V, q.sigma[: q.k])
    assert mt["sigma_err"] <= 1e-12 and mt["residV"] <= 1e-13 and mt["residU"] <= 1e-13, mt
