"""GPU parity of the full-spectrum QDWH-SVD (Section 3.2) through the C ABI:
qdwhp_gesvd_f64 against the definition (every singular triplet: constructed singular
values, the oracle's qdwh_svd and the LAPACK SVD) at the plain-FP64 tolerances
|sigma - sigma*| <= 1e-12 ||A||_2, ||U^T U - I||_F, ||V^T V - I||_F <= 5e-15 p,
||A V - U Sigma||_F / ||A||_F and ||A^T U - V Sigma||_F / ||A||_F <= 1e-13."""

import numpy as np
import pytest

import oracle as O
from paper_2104_14186_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SIG_TOL = 1e-12
ORTH_TOL = 5e-15
RES_TOL = 1e-13


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


def check(A, s, U, V, s_true):
    m, n = A.shape
    p = min(m, n)
    s, U, V = s.cpu().numpy(), U.cpu().numpy(), V.cpu().numpy()
    assert s.shape == (p,) and U.shape == (m, p) and V.shape == (n, p)
    assert np.all(np.diff(s) <= 0)
    mt = O.svd_metrics(A, s, U, V, s_true)
    assert mt["sigma_err"] <= SIG_TOL, mt
    assert mt["orthU"] <= ORTH_TOL * p and mt["orthV"] <= ORTH_TOL * p, mt
    assert mt["residV"] <= RES_TOL and mt["residU"] <= RES_TOL, mt
    return mt


def problem(m, n, seed):
    """sigma log-spaced over 12 decades; m < n by transposing the m >= n construction."""
    if m >= n:
        p = I.svd_logspaced(m, n, seed)
        return p.A, p.sigma
    p = I.svd_logspaced(n, m, seed)
    return np.asfortranarray(p.A.T), p.sigma


@pytest.mark.parametrize("m,n", [(1, 1), (6, 1), (1, 6), (40, 25), (25, 40), (300, 300), (513, 400),
                                 (700, 600), (600, 700)])
def test_gesvd_constructed(Q, m, n):
    """Leaf-only (p <= 512) and divide-and-conquer (p > 512) eigensolves of H, tall and wide."""
    A, sig = problem(m, n, 100 + m + n)
    s, U, V, info = Q.gesvd(dev(A))
    check(A, s, U, V, sig)
    assert info["orthonormalized"] == 0, info
    if min(m, n) > 1:
        assert info["it_qr"] >= 1 and info["it_qr"] + info["it_chol"] == 6, info
    if min(m, n) > 512:
        assert info["nodes"] >= 1, info


def test_gesvd_matches_oracle(Q):
    """Element by element against the oracle's QDWH-SVD and the LAPACK SVD (random A)."""
    rng = np.random.default_rng(17)
    A = rng.standard_normal((260, 210))
    s, U, V, _ = Q.gesvd(dev(A))
    s = s.cpu().numpy()
    so, _, _, _ = O.full.qdwh_svd(A)
    sd, _, _ = O.full.gesvd(A)
    assert np.max(np.abs(s - so)) <= SIG_TOL * sd[0]
    assert np.max(np.abs(s - sd)) <= SIG_TOL * sd[0]
    check(A, torch.from_numpy(s), U, V, sd)


def test_gesvd_rank_deficient(Q):
    """60 exact zero singular values: U is completed orthonormally and flagged."""
    rng = np.random.default_rng(23)
    sig = np.concatenate([np.sort(rng.uniform(0.5, 2.0, 340))[::-1], np.zeros(60)])
    A = I.general_with_singular_values(500, sig, rng)
    s, U, V, info = Q.gesvd(dev(A))
    check(A, s, U, V, sig)
    assert info["orthonormalized"] == 1, info


def test_gesvd_paper_graded_spectrum(Q):
    """The paper's test spectrum D[i] = 0.5^(100 i / n) (condition ~1e30, beyond the polar
    factor's ell_0): singular values to 1e-12 ||A||, U completed on the unsettled directions."""
    p = I.svd_geometric_half(400, 29)
    s, U, V, info = Q.gesvd(dev(p.A))
    check(p.A, s, U, V, p.sigma)
    assert info["orthonormalized"] == 1, info


def test_gesvd_zero_and_nonfinite(Q):
    s, U, V, info = Q.gesvd(dev(np.zeros((300, 200))))
    assert torch.all(s == 0)
    assert torch.equal(U.cpu(), torch.eye(300, 200, dtype=torch.float64))
    assert torch.equal(V.cpu(), torch.eye(200, dtype=torch.float64))
    A = np.eye(300, 200)
    A[4, 9] = np.inf
    with pytest.raises(Q.QdwhpError) as e:
        Q.gesvd(dev(A))
    assert e.value.status == -5


@pytest.mark.parametrize("m,n", [(1024, 1024), (700, 600)])
def test_gesvd_emulated(Q, m, n):
    """FP64 products emulated on the BF16 tensor cores: the same FP64 tolerances."""
    A, sig = problem(m, n, 7 + m)
    s, U, V, info = Q.gesvd(dev(A), precision=Q.FP64_EMULATED)
    check(A, s, U, V, sig)
