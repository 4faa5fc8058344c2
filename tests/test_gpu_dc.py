"""GPU parity of the QDWH spectral divide-and-conquer eigensolver (QDWH-EIG, Section 3.2),
through the C ABI: qdwhp_syev_f64 against the definition (all eigenpairs of the symmetric
matrix: the oracle's syev and the constructed spectrum), and the partial EIG solver on
problems whose Rayleigh-Ritz step is large enough to take the divide-and-conquer route.
Tolerances are the plain-FP64 ones: |lambda - lambda*| <= 1e-12 ||A||_2,
||V^T V - I||_F <= 5e-15 n, ||A V - V Lambda||_F / ||A||_F <= 1e-13."""

import numpy as np
import pytest

import oracle as O
from paper_2104_14186_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LAM_TOL = 1e-12
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


def check_full(A, lam_true, lam, V):
    n = A.shape[0]
    lam, V = lam.cpu().numpy(), V.cpu().numpy()
    assert np.all(np.diff(lam) >= 0)
    m = O.eig_metrics(A, lam, V, np.sort(lam_true))
    assert m["lam_err"] <= LAM_TOL, m
    assert m["orth"] <= ORTH_TOL * n, m
    assert m["resid"] <= RES_TOL, m
    ref, _ = O.syev(A)
    assert np.max(np.abs(lam - ref)) <= LAM_TOL * np.max(np.abs(lam_true))
    return m


@pytest.mark.parametrize("n,seed", [(1, 1), (2, 2), (300, 3), (512, 4), (513, 5), (1100, 6), (1537, 7)])
def test_syev_uniform(Q, n, seed):
    """Leaf-only (n <= 512) and split (one and two levels) cases, ragged sizes."""
    rng = np.random.default_rng(seed)
    lam = rng.uniform(-1.0, 1.0, n)
    A = I.symmetric_with_spectrum(lam, rng)
    l, V, info = Q.syev(dev(A))
    check_full(A, lam, l, V)
    if n > 512:
        assert info["nodes"] >= 1 and info["leaves"] >= 2, info
        assert info["max_offblock"] <= 1e-12, info
    else:
        assert info["nodes"] == 0


def test_syev_clusters_and_multiplicities(Q):
    """Exact multiplicities, a 1e-10-wide cluster and a split point that may fall inside a
    cluster: every eigenpair still meets the tolerances."""
    rng = np.random.default_rng(11)
    n = 1300
    lam = np.concatenate([rng.uniform(-1, 1, 700), np.full(300, 0.1), 0.6 + 1e-10 * rng.standard_normal(300)])
    A = I.symmetric_with_spectrum(lam, rng)
    l, V, info = Q.syev(dev(A))
    check_full(A, lam, l, V)


def test_syev_graded_unbalanced(Q):
    """A graded positive spectrum (1e-8 .. 1): the mean sits near the top, so the splits
    are unbalanced and the recursion deepens."""
    rng = np.random.default_rng(13)
    n = 1200
    lam = 10.0 ** rng.uniform(-8, 0, n)
    A = I.symmetric_with_spectrum(lam, rng)
    l, V, info = Q.syev(dev(A))
    check_full(A, lam, l, V)
    assert info["depth"] >= 2, info


def test_syev_nonfinite_input(Q):
    A = np.eye(600)
    A[5, 7] = np.nan
    with pytest.raises(Q.QdwhpError) as e:
        Q.syev(dev(A))
    assert e.value.status == -5


@pytest.mark.parametrize("frac,side", [(0.45, "largest"), (0.40, "smallest")])
def test_partial_eig_takes_divide_and_conquer(Q, frac, side):
    """n = 2400 with 40-45 % wanted: the Rayleigh-Ritz problem (ell > 1024) is solved by
    divide and conquer; the k pairs meet the plain-FP64 tolerances."""
    p = I.eig_uniform(2400, 77, frac, side)
    r = Q.eig(dev(p.A), k=p.k, side=side)
    assert r.info["ell"] > 1024 and r.info["dc_nodes"] >= 1, r.info
    lam, V = r.lam.cpu().numpy(), r.V.cpu().numpy()
    true = np.sort(p.lam)[::-1][: p.k] if side == "largest" else np.sort(p.lam)[: p.k]
    m = O.eig_metrics(p.A, lam, V, true)
    assert m["lam_err"] <= LAM_TOL, m
    assert m["orth"] <= ORTH_TOL * 2400, m
    assert m["resid"] <= RES_TOL, m


@pytest.mark.parametrize("c", [0.0, 1.5])
def test_syev_one_point_spectrum(Q, c):
    """c I (and the zero matrix) through the divide-and-conquer solver: every eigenvalue c,
    orthonormal vectors."""
    n = 700
    lam, V, info = Q.syev(dev(c * np.eye(n)))
    lam, V = lam.cpu().numpy(), V.cpu().numpy()
    assert np.max(np.abs(lam - c)) <= 1e-14 * max(1.0, abs(c))
    assert np.linalg.norm(V.T @ V - np.eye(n)) <= ORTH_TOL * n


def test_syev_graded_splits_at_quadrature_median(Q):
    """Eigenvalues log-spaced over 12 decades (n = 1500): the splits are made at the Lanczos
    quadrature estimate of the median, depth 3 (at the mean eigenvalue each split peels off
    ~12 % and the depth is 7); every eigenpair meets the tolerances."""
    rng = np.random.default_rng(17)
    lam = 10.0 ** (-12.0 * np.arange(1500) / 1499)
    A = I.symmetric_with_spectrum(lam, rng)
    l, V, info = Q.syev(dev(A))
    check_full(A, lam, l, V)
    assert info["median_splits"] >= 2 and info["depth"] <= 4, info


def test_syev_two_point_spectrum(Q):
    """Two eigenvalues, 100-fold and 900-fold: one split separates them exactly."""
    rng = np.random.default_rng(19)
    lam = np.concatenate([np.full(100, -0.5), np.full(900, 2.0)])
    A = I.symmetric_with_spectrum(lam, rng)
    l, V, info = Q.syev(dev(A))
    check_full(A, lam, l, V)
    assert info["nodes"] == 1, info
