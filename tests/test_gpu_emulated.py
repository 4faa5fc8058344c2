"""FP64 products emulated on the BF16 tensor cores (Ozaki splitting), through the C ABI.

The emulated GEMM is checked against its definition (the numpy FP64 product) with the
scheme's error bound: the inputs are rounded to 53 bits relative to the largest entry of
each row of op(A) and column of op(B), the digit pairs with s + t > 12 (each term at most 2^-64
of the row maximum times the column maximum) are dropped, and the 60 exact partial products
are summed in FP64.  The solvers in QDWHP_FP64_EMULATED mode must
meet the plain-FP64 tolerances: |lambda - lambda*| <= 1e-12 ||A||_2,
||V^T V - I||_F <= 5e-15 n, residuals <= 1e-13."""

import numpy as np
import pytest

import oracle as O
from paper_2104_14186_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

U64 = 2.0 ** -53


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


def emulation_bound(opA, opB, alpha, beta, C0):
    k = opA.shape[1]
    absA, absB = np.abs(opA), np.abs(opB)
    scale = abs(alpha) * (absA @ absB) + abs(beta) * np.abs(C0)
    rowmax = absA.max(axis=1, initial=0.0)[:, None]
    colmax = absB.max(axis=0, initial=0.0)[None, :]
    trunc = abs(alpha) * 2.0 ** -52 * (rowmax * absB.sum(axis=0)[None, :] + colmax * absA.sum(axis=1)[:, None])
    dropped = abs(alpha) * 1e-16 * k * rowmax * colmax
    # (4 k + 64) u |A||B|: the FP64 reference's own rounding plus the FP64 sum of the digit products
    return (4 * k + 64) * U64 * scale + trunc + dropped + 1e-300


@pytest.mark.parametrize("m,n,k", [(128, 128, 256), (300, 257, 1000), (37, 530, 300), (130, 200, 9000),
                                   (512, 512, 512)])
@pytest.mark.parametrize("ta,tb", [(False, False), (False, True), (True, False), (True, True)])
def test_emulated_gemm_within_bound(Q, m, n, k, ta, tb):
    rng = np.random.default_rng(m * 11 + n * 5 + k + 2 * ta + tb)
    A = rng.standard_normal((k, m) if ta else (m, k))
    B = rng.standard_normal((n, k) if tb else (k, n))
    A[3] *= 1e-8            # rows and columns of very different magnitude
    B[:, 5] *= 1e6
    C0 = rng.standard_normal((m, n))
    opA, opB = (A.T if ta else A), (B.T if tb else B)
    ref = 1.5 * opA @ opB - 0.5 * C0
    got = Q.gemm_f64_emulated(dev(A), dev(B), ta, tb, alpha=1.5, beta=-0.5, Cmat=dev(C0)).cpu().numpy()
    err = np.abs(got - ref)
    bound = emulation_bound(opA, opB, 1.5, -0.5, C0)
    assert np.all(err <= bound), float(np.max(err / bound))
    # and it agrees with the native FP64 product to FP64 accuracy, normwise
    nat = Q.gemm_f64(dev(A), dev(B), ta, tb, alpha=1.5, beta=-0.5, Cmat=dev(C0)).cpu().numpy()
    assert np.linalg.norm(got - nat) <= 1e-14 * np.linalg.norm(np.abs(opA) @ np.abs(opB))


def test_emulated_gemm_exact_on_integers_with_digit_carries(Q):
    """Integer entries below 2^20 whose 6-bit groups are 63 or 32 (every balanced digit carries,
    the top digit reaches its bound 32): the digits hold them exactly and no kept pair is
    dropped, so the emulated product equals the exact integer product."""
    rng = np.random.default_rng(11)
    m, k, n = 200, 300, 136
    pool = np.array([2 ** 20 - 1, 2 ** 19 + 2 ** 13 - 1, 0b100000_100000_100000, 2 ** 18 + 1, 63, 32])
    A = (rng.choice(pool, (m, k)) * rng.choice([-1, 1], (m, k))).astype(np.int64)
    B = (rng.choice(pool, (k, n)) * rng.choice([-1, 1], (k, n))).astype(np.int64)
    A[:, 0] = 2 ** 20 - 1                     # every row's largest entry: all ones
    exact = A @ B                             # |entries| < 300 * 2^40: exact in int64 and FP64
    got = Q.gemm_f64_emulated(dev(A.astype(np.float64)), dev(B.astype(np.float64))).cpu().numpy()
    assert np.array_equal(got, exact.astype(np.float64))


def test_emulated_gemm_all_ones_mantissas(Q):
    """Entries +-(1 - 2^-53) 2^p: the 53-bit integer of a row's largest entry is 2^53 - 1, so every
    6-bit group is 63 and the carry reaches the top digit."""
    rng = np.random.default_rng(12)
    m, k, n = 160, 520, 140
    A = rng.choice([-1.0, 1.0], (m, k)) * (1 - 2.0 ** -53) * 2.0 ** rng.integers(-3, 1, (m, k))
    B = rng.choice([-1.0, 1.0], (k, n)) * (1 - 2.0 ** -53) * 2.0 ** rng.integers(-3, 1, (k, n))
    got = Q.gemm_f64_emulated(dev(A), dev(B)).cpu().numpy()
    ref = A @ B
    assert np.all(np.abs(got - ref) <= emulation_bound(A, B, 1.0, 0.0, np.zeros_like(ref)))


def test_emulated_gemm_k_beyond_one_launch(Q):
    """K = 66000 exceeds one digit-product schedule (65536 deep): the product runs as two
    launches, the second adding onto C."""
    rng = np.random.default_rng(13)
    m, k, n = 130, 66000, 128
    A = rng.standard_normal((m, k))
    B = rng.standard_normal((k, n))
    C0 = rng.standard_normal((m, n))
    got = Q.gemm_f64_emulated(dev(A), dev(B), alpha=1.5, beta=-0.5, Cmat=dev(C0)).cpu().numpy()
    ref = 1.5 * A @ B - 0.5 * C0
    assert np.all(np.abs(got - ref) <= emulation_bound(A, B, 1.5, -0.5, C0))


def test_emulated_gemm_zero_and_nonfinite_rows(Q):
    rng = np.random.default_rng(3)
    A = rng.standard_normal((200, 300))
    B = rng.standard_normal((300, 150))
    A[7] = 0.0
    A[9, 4] = np.nan
    got = Q.gemm_f64_emulated(dev(A), dev(B)).cpu().numpy()
    assert np.all(got[7] == 0.0)
    assert np.all(np.isnan(got[9]))
    ok = np.ones(200, bool)
    ok[[7, 9]] = False
    assert np.all(np.isfinite(got[ok]))
    ref = A[ok] @ B
    assert np.all(np.abs(got[ok] - ref) <= emulation_bound(A[ok], B, 1.0, 0.0, np.zeros_like(ref)))


def test_emulated_gemm_beta_zero_ignores_nan_in_c(Q):
    A = np.eye(256)
    C0 = np.full((256, 256), np.nan)
    got = Q.gemm_f64_emulated(dev(A), dev(A), beta=0.0, Cmat=dev(C0)).cpu().numpy()
    assert np.array_equal(got, np.eye(256))


def test_emulated_eig_workload_n512(Q):
    p = I.eig_uniform(512, 1000, 0.10)
    r = Q.eig(dev(p.A), k=p.k, precision=Q.FP64_EMULATED)
    m = O.eig_metrics(p.A, r.lam.cpu().numpy(), r.V.cpu().numpy(), np.sort(p.lam)[::-1][: p.k])
    assert m["lam_err"] <= 1e-12 and m["orth"] <= 5e-15 * 512 and m["resid"] <= 1e-13, m


@pytest.mark.parametrize("m,n,frac,seed", [(700, 500, 0.05, 2000), (4096, 4096, 0.05, 2000)])
def test_emulated_svd(Q, m, n, frac, seed):
    q = I.svd_logspaced(m, n, seed, frac)
    r = Q.svd(dev(q.A), k=q.k, precision=Q.FP64_EMULATED)
    mt = O.svd_metrics(q.A, r.sigma.cpu().numpy(), r.U.cpu().numpy(), r.V.cpu().numpy(), q.sigma[: q.k])
    assert mt["sigma_err"] <= 1e-12, mt
    assert mt["orthU"] <= 5e-15 * n and mt["orthV"] <= 5e-15 * n, mt
    assert mt["residV"] <= 1e-13 and mt["residU"] <= 1e-13, mt


@pytest.mark.parametrize("m,n,frac,seed", [(1500, 1000, 0.20, 3), (2000, 1200, 0.15, 4)])
def test_emulated_svd_with_a_qr_based_step(Q, m, n, frac, seed):
    """The serving stream's SVD shape: sigma over 10 decades and 15-20 % wanted put s near 1e-2,
    so the schedule starts with a QR-based step (c_0 > 100), whose reductions run emulated."""
    q = I.svd_logspaced(m, n, seed, frac, decades=10.0)
    r = Q.svd(dev(q.A), k=q.k, precision=Q.FP64_EMULATED)
    assert r.info["it_qr"] >= 1
    mt = O.svd_metrics(q.A, r.sigma.cpu().numpy(), r.U.cpu().numpy(), r.V.cpu().numpy(), q.sigma[: q.k])
    print(f"{m}x{n} {frac}: {mt}")
    assert mt["sigma_err"] <= 1e-12, mt
    assert mt["orthU"] <= 5e-15 * m and mt["orthV"] <= 5e-15 * m, mt
    assert mt["residV"] <= 1e-13 and mt["residU"] <= 1e-13, mt


def test_mixed_emulated_svd_refined_meets_fp64_tolerances(Q):
    """FP32 Cholesky steps, emulated FP64 products elsewhere and 6 FP64 subspace-refinement
    steps: the SVD workload (4096 x 4096, top 5 %) at the plain-FP64 tolerances."""
    q = I.svd_logspaced(4096, 4096, 2000, 0.05)
    r = Q.svd(dev(q.A), k=q.k, precision=Q.MIXED_EMULATED, refine_steps=6)
    assert r.info["it_f32"] == 2
    mt = O.svd_metrics(q.A, r.sigma.cpu().numpy(), r.U.cpu().numpy(), r.V.cpu().numpy(), q.sigma[: q.k])
    assert mt["sigma_err"] <= 1e-12, mt
    assert mt["orthU"] <= 5e-15 * 4096 and mt["orthV"] <= 5e-15 * 4096, mt
    assert mt["residV"] <= 1e-13 and mt["residU"] <= 1e-13, mt
