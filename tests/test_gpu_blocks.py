"""GPU parity of the dense building blocks (through the C ABI) against FP64 references:
numpy products, the oracle's QDWH steps and the spectral-map identity."""

import numpy as np
import pytest

import oracle as O
from paper_2104_14186_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def Q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_14186_gb300 import build
    build.build()
    from paper_2104_14186_gb300 import qdwhp
    return qdwhp


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (37, 53, 71), (64, 64, 64), (200, 130, 300), (33, 1000, 17),
                                   (512, 512, 512), (32, 96, 5000)])
@pytest.mark.parametrize("ta,tb", [(False, False), (False, True), (True, False), (True, True)])
def test_gemm(Q, m, n, k, ta, tb):
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    A = rng.standard_normal((k, m) if ta else (m, k))
    B = rng.standard_normal((n, k) if tb else (k, n))
    C0 = rng.standard_normal((m, n))
    ref = 1.5 * (A.T if ta else A) @ (B.T if tb else B) - 0.5 * C0
    got = Q.gemm_f64(dev(A), dev(B), ta, tb, alpha=1.5, beta=-0.5, Cmat=dev(C0)).cpu().numpy()
    scale = 1.5 * np.abs(A if not ta else A.T) @ np.abs(B if not tb else B.T) + 0.5 * np.abs(C0)
    assert np.all(np.abs(got - ref) <= 4 * k * 2.0 ** -53 * scale + 1e-300)


def test_gemm_beta_zero_ignores_nan_in_c(Q):
    A = np.eye(8)
    C0 = np.full((8, 8), np.nan)
    got = Q.gemm_f64(dev(A), dev(A), beta=0.0, Cmat=dev(C0)).cpu().numpy()
    assert np.array_equal(got, np.eye(8))


@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 200, 513, 1100])
def test_potrf(Q, n):
    rng = np.random.default_rng(n)
    G = rng.standard_normal((n, n))
    Z = G @ G.T / n + np.eye(n)
    L, info = Q.potrf_f64(dev(Z))
    L = L.cpu().numpy()
    assert info == 0
    ref = np.linalg.cholesky(Z)
    assert np.linalg.norm(L - ref) <= 1e-13 * np.linalg.norm(ref) * max(1, np.sqrt(n) / 10)
    assert np.linalg.norm(L @ L.T - Z) <= 1e-14 * n * np.linalg.norm(Z)


def test_potrf_reports_breakdown(Q):
    n = 150
    Z = np.eye(n)
    Z[100, 100] = -1.0
    _, info = Q.potrf_f64(dev(Z))
    assert info == 101


@pytest.mark.parametrize("m,n", [(1, 1), (5, 3), (70, 64), (100, 37), (300, 300), (1000, 200), (777, 129)])
def test_qr(Q, m, n):
    rng = np.random.default_rng(m + 1000 * n)
    A = rng.standard_normal((m, n))
    Qm, R = Q.qr_f64(dev(A))
    Qm, R = Qm.cpu().numpy(), R.cpu().numpy()
    assert np.allclose(np.tril(R, -1), 0.0)
    assert np.linalg.norm(Qm.T @ Qm - np.eye(n)) <= 1e-14 * n
    assert np.linalg.norm(Qm @ R - A) <= 1e-14 * n * np.linalg.norm(A)
    Rref = np.linalg.qr(A, mode="r")
    # the Householder R is unique up to the signs of its rows
    assert np.allclose(np.abs(np.diag(R)), np.abs(np.diag(Rref)), rtol=1e-12, atol=1e-12)
    # same sign convention as LAPACK: R_ii = -sign(a_ii) ||.||
    assert np.array_equal(np.sign(np.diag(R)), np.sign(np.diag(Rref)))


def test_qr_rank_deficient(Q):
    """The extraction QR runs on (nearly) rank-deficient matrices: a projector of rank 40."""
    rng = np.random.default_rng(5)
    n = 160
    U = I.haar_orthogonal(n, rng)[:, :40]
    P = U @ U.T
    Qm, R = Q.qr_f64(dev(P))
    Qm, R = Qm.cpu().numpy(), R.cpu().numpy()
    assert np.linalg.norm(Qm.T @ Qm - np.eye(n)) <= 1e-13 * n
    assert np.linalg.norm(Qm @ R - P) <= 1e-13 * n
    d = np.abs(np.diag(R))
    assert np.all(d[:40] > 0.01) and np.all(d[40:] < 1e-10)


def test_qdwh_chol_steps_match_oracle_and_spectral_map(Q):
    rng = np.random.default_rng(3)
    n = 300
    lam = np.concatenate([rng.uniform(-1, -0.2, 40), rng.uniform(-0.2, 6.0, n - 40)])
    Qh = I.haar_orthogonal(n, rng)
    X0 = (Qh * lam) @ Qh.T
    sched = O.dwh_schedule(0.2, fixed_iters=3)
    Xg, conv = Q.qdwh_steps_f64(dev(X0), [s[:3] for s in sched], [0, 0, 0])
    Xg = Xg.cpu().numpy()
    Xo = X0.copy()
    y = lam.copy()
    for a, b, c, _, _ in sched:
        Xprev = Xo
        Xo = O.qdwh_chol_step(Xo, a, b, c)
        y = O.rational_map(y, a, b, c)
    ref = (Qh * y) @ Qh.T
    assert np.linalg.norm(Xg - Xo) <= 1e-13 * np.linalg.norm(Xo)
    assert np.linalg.norm(Xg - ref) <= 1e-13 * np.linalg.norm(ref)
    assert abs(conv[-1] - np.linalg.norm(Xo - Xprev)) <= 1e-10 * max(1.0, conv[-1])


@pytest.mark.parametrize("m,n", [(260, 190), (700, 600), (600, 600), (1100, 520)])
def test_qdwh_qr_step_matches_oracle(Q, m, n):
    """QR-based steps (the stacked [sqrt(c) X; I] factored with its identity block's zeros
    skipped) against the oracle's dense QR step and the spectral map, over one and several
    256-column outer blocks, ragged and square."""
    rng = np.random.default_rng(4 + m + n)
    sig = np.geomspace(1.0, 1e-3, n)
    U = I.haar_orthogonal(n, rng, m)
    V = I.haar_orthogonal(n, rng)
    X0 = (U * sig) @ V.T
    sched = O.dwh_schedule(1e-3)
    use_qr = [1 if s[2] > 100 else 0 for s in sched]
    assert use_qr[0] == 1
    Xg, _ = Q.qdwh_steps_f64(dev(X0), [s[:3] for s in sched], use_qr)
    Xg = Xg.cpu().numpy()
    y = sig.copy()
    Xo = X0.copy()
    for (a, b, c, _, _), uq in zip(sched, use_qr):
        Xo = O.qdwh_qr_step(Xo, a, b, c) if uq else O.qdwh_chol_step(Xo, a, b, c)
        y = O.rational_map(y, a, b, c)
    ref = (U * y) @ V.T
    assert np.linalg.norm(Xg - Xo) <= 1e-12 * np.linalg.norm(Xo)
    assert np.linalg.norm(Xg - ref) <= 1e-12 * np.linalg.norm(ref)
