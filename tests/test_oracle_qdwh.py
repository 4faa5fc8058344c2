"""Pins of the oracle's QDWH building blocks against facts fixed by the paper
and by mathematics (not against the oracle itself)."""

import math

import numpy as np
import pytest

import oracle as O
from conftest import golden
from paper_2104_14186_gb300 import inputs as I

G = golden("paper_values.txt")


def _count_to_convergence(ell0):
    return len(O.dwh_schedule(ell0))


def test_iteration_counts_printed_in_paper():
    # Section 3.1: at most six iterations for kappa <= 1e15.
    assert _count_to_convergence(1e-15) <= int(G["qdwh_max_iters_kappa_1e15"])
    for ell0 in np.logspace(-15, -0.01, 60):
        assert _count_to_convergence(ell0) <= int(G["qdwh_max_iters_kappa_1e15"])
    # Section 4.1: three iterations for s = 0.2, two for s = 0.875 reach O(u) on [-1, 0].
    for s, key in ((0.2, "eig_iters_s_0.2"), (0.875, "eig_iters_s_0.875")):
        it = int(G[key])
        sch = O.dwh_schedule(s, fixed_iters=it)
        x = np.linspace(-1.0, 0.0, 20001)
        y = (1.0 - s) * x - s
        for a, b, c, _, _ in sch:
            y = O.rational_map(y, a, b, c)
        assert np.max(np.abs(y + 1.0)) < 20 * 2.0 ** -53   # O(u)
        # ... and one iteration fewer does not
        y = (1.0 - s) * x - s
        for a, b, c, _, _ in sch[:-1]:
            y = O.rational_map(y, a, b, c)
        assert np.max(np.abs(y + 1.0)) > 1e-9


def test_band_where_r_plus_one_is_order_one():
    # Section 4.1: with three iterations (s = 0.2) r(x)+1 is O(1) from x ~ 0.1 on;
    # with two iterations (s = 0.875) only from x ~ 5.
    for s, it, key in ((0.2, 3, "eig_band_three_iters_x"), (0.875, 2, "eig_band_two_iters_x")):
        x_paper = float(G[key])
        sch = O.dwh_schedule(s, fixed_iters=it)
        x = np.linspace(0.0, 20.0, 200001)
        y = (1.0 - s) * x - s
        for a, b, c, _, _ in sch:
            y = O.rational_map(y, a, b, c)
        x_on = x[np.argmax(0.5 * (y + 1.0) >= 0.01)]
        assert 0.5 * x_paper <= x_on <= 2.5 * x_paper


@pytest.mark.parametrize("ell", [0.9, 0.5, 0.2, 0.05, 1e-2, 1e-3, 1e-6, 1e-10, 1e-15])
def test_weights_are_the_optimal_type_32_function(ell):
    """The DWH weights make r(x) = x(a+bx^2)/(1+cx^2) the best (3,2) approximation
    of sign on [ell, 1]: r <= 1 on [ell, 1], r(1) = 1 and r = 1 at an interior
    critical point (equioscillation), minimum at x = ell where it equals ell_next."""
    a, b, c, ell_next = O.dwh_weights(ell)
    assert abs(c - (a + b - 1.0)) <= 1e-15 * c          # r(1) = 1
    x = np.concatenate([np.geomspace(ell, 1.0, 400001)])
    y = O.rational_map(x, a, b, c)
    assert y.max() <= 1.0 + 1e-13
    assert abs(y[0] - ell_next) <= 1e-14 * max(ell_next, 1e-300) + 1e-300
    assert np.argmin(y) == 0
    # interior maximum: r'(x) = 0 at x*^2 solving b c x^4 + (3b - a c) x^2 + a = 0, with r(x*) = 1
    disc = (3 * b - a * c) ** 2 - 4 * b * c * a
    x2 = ((a * c - 3 * b) - math.sqrt(max(disc, 0.0))) / (2 * b * c)
    xs = math.sqrt(x2)
    assert ell < xs <= 1.0 + 1e-6
    assert abs(O.rational_map(xs, a, b, c) - 1.0) <= 1e-9
    # optimality: no perturbed (3,2) function has a larger min/max ratio on [ell, 1]
    # (the DWH function attains ratio ell_next)
    rng = np.random.default_rng(int(-math.log10(ell) * 10))
    for _ in range(20):
        a2 = a * (1 + 0.05 * rng.standard_normal())
        b2 = b * (1 + 0.05 * rng.standard_normal())
        c2 = c * (1 + 0.05 * rng.standard_normal())
        if min(a2, b2, c2) <= 0:
            continue
        y2 = O.rational_map(x, a2, b2, c2)
        assert y2.min() / y2.max() <= ell_next * (1 + 1e-9)


def _scalar_chain(x, sched):
    for a, b, c, _, _ in sched:
        x = O.rational_map(x, a, b, c)
    return x


def test_chol_step_spectral_map_symmetric():
    """X_k = Q r_k(...r_1(lam)) Q^T for A = Q diag(lam) Q^T (every iterate is a function of A)."""
    rng = np.random.default_rng(7)
    n = 96
    lam = np.concatenate([rng.uniform(-1, -0.2, 30), rng.uniform(-0.2, 6.0, 66)])
    Q = I.haar_orthogonal(n, rng)
    X = (Q * lam) @ Q.T
    sched = O.dwh_schedule(0.2, fixed_iters=3)
    y = lam.copy()
    for a, b, c, _, _ in sched:
        X = O.qdwh_chol_step(X, a, b, c)
        y = O.rational_map(y, a, b, c)
        ref = (Q * y) @ Q.T
        assert np.linalg.norm(X - ref) <= 1e-13 * np.linalg.norm(ref)


@pytest.mark.parametrize("m,n", [(70, 50), (50, 50)])
def test_qr_and_chol_steps_spectral_map_rectangular(m, n):
    """For X = U diag(sig) V^T both step forms give U diag(r(sig)) V^T (eq. practical-polar-qr
    and eq. practical-polar-chol are the same iteration)."""
    rng = np.random.default_rng(m + n)
    sig = np.geomspace(1.0, 1e-3, n)
    U = I.haar_orthogonal(n, rng, m)
    V = I.haar_orthogonal(n, rng)
    X0 = (U * sig) @ V.T
    sched = O.dwh_schedule(1e-3)
    Xq = X0.copy()
    Xc = X0.copy()
    y = sig.copy()
    for i, (a, b, c, _, _) in enumerate(sched):
        Xq = O.qdwh_qr_step(Xq, a, b, c)
        y = O.rational_map(y, a, b, c)
        ref = (U * y) @ V.T
        assert np.linalg.norm(Xq - ref) <= 1e-12 * np.linalg.norm(ref), i
        if i >= 1:  # the Cholesky form from the second step on (c_k small)
            Xc = O.qdwh_chol_step(Xc, a, b, c)
            assert np.linalg.norm(Xc - ref) <= 1e-11 * np.linalg.norm(ref), i
        else:
            Xc = Xq.copy()


@pytest.mark.parametrize("kappa", [1e4, 1e8])
def test_polar_factor_against_svd(kappa):
    """QDWH converges to the polar factor U V^T; its forward error is O(u kappa)."""
    rng = np.random.default_rng(3)
    m, n = 90, 60
    sig = np.geomspace(2.0, 2.0 / kappa, n)
    U = I.haar_orthogonal(n, rng, m)
    V = I.haar_orthogonal(n, rng)
    A = (U * sig) @ V.T
    Up, H, sched = O.qdwh_polar(A, alpha=2.0, ell0=0.9 / kappa)
    assert len(sched) <= 6
    Uu, ss, Vt = np.linalg.svd(A, full_matrices=False)
    assert np.linalg.norm(Up - Uu @ Vt) <= 50 * 2.0 ** -53 * kappa * math.sqrt(n)
    assert np.linalg.norm(Up.T @ Up - np.eye(n)) <= 1e-13 * n
    assert np.linalg.norm(H - H.T) == 0.0
    assert np.linalg.eigvalsh(H).min() >= -1e-12
    assert np.linalg.norm(Up @ H - A) <= 1e-12 * np.linalg.norm(A)


def test_splitmix64_published_outputs():
    ref = [int(line, 16) for line in open(__file__.replace("test_oracle_qdwh.py", "golden/splitmix64.txt"))
           if line.startswith("0x")]
    got = [int(v) for v in O.splitmix64(0, 3)]
    assert got == ref
    u = O.uniform_pm1(99, 200000)
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 0.01 and abs(u.var() - 1.0 / 3.0) < 0.01
    assert np.array_equal(O.uniform_pm1(99, 10, offset=5), u[5:15])
