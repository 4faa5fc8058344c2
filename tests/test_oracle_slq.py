"""Pins of the oracle's stochastic Lanczos quadrature threshold (the count-to-threshold
estimate for wide blocks): the Gauss rule of the Lanczos tridiagonal, the lower bound of a
spectral distribution read off it, and the threshold it gives on constructed spectra."""

import numpy as np
import pytest

import oracle as O
from paper_2104_14186_gb300 import inputs as I
from oracle.partial import STREAM_LANCZOS, slq_probe_seed
from oracle.rng import uniform_pm1


def _probe(A, steps, seed):
    n = A.shape[0]
    al, be = O.lanczos_tridiagonal(lambda x: A @ x, n, steps, seed)
    v = uniform_pm1(seed ^ STREAM_LANCZOS, n)
    return O.gauss_rule(al, be), v / np.linalg.norm(v)


@pytest.mark.parametrize("steps", [5, 12, 30, 64])
def test_gauss_rule_exact_for_low_degree(steps):
    """An m-node Gauss rule integrates x^d exactly for d <= 2m - 1: sum_i w_i theta_i^d =
    v^T A^d v for the unit start vector v (a dropped square of the weights, a missing
    normalisation or a wrong node would break this)."""
    rng = np.random.default_rng(steps)
    n = 200
    lam = rng.uniform(-1, 1, n)
    A = I.symmetric_with_spectrum(lam, rng)
    (theta, w), v = _probe(A, steps, 31 + steps)
    assert abs(w.sum() - 1.0) < 1e-13
    Av = v.copy()
    for d in range(1, min(2 * steps - 1, 24) + 1):
        Av = A @ Av
        assert abs(np.sum(w * theta ** d) - v @ Av) <= 1e-11, d


@pytest.mark.parametrize("steps", [5, 12, 30, 64])
def test_lower_bound_never_exceeds_the_distribution(steps):
    """Chebyshev-Markov-Stieltjes: at every point x (the nodes, points between them, beyond
    them) the lower bound read off the Gauss rule is at most the probe's exact spectral
    distribution F_v(x) = sum of (v^T u_i)^2 over lambda_i <= x, on continuous spectra."""
    for trial in range(6):
        rng = np.random.default_rng(100 + trial)
        n = 300
        lam = rng.uniform(-1, 1, n) if trial % 2 else np.concatenate([rng.uniform(-1, -0.4, 200),
                                                                        rng.uniform(0.6, 1.0, 100)])
        A = I.symmetric_with_spectrum(lam, rng)
        lamA, U = np.linalg.eigh(A)
        (theta, w), v = _probe(A, steps, 7 + trial)
        mu = (U.T @ v) ** 2
        xs = np.concatenate([theta, 0.5 * (theta[1:] + theta[:-1]), [theta[0] - 1, theta[-1] + 1],
                             np.linspace(-1.2, 1.2, 97)])
        for x in xs:
            F = mu[lamA <= x].sum()
            assert O.slq_lower_bound(theta, w, x) <= F + 1e-12, (x, F)
        # and it is not vacuous: just above the largest node it is 1 - w_last
        assert O.slq_lower_bound(theta, w, theta[-1] + 1e-9) == pytest.approx(1.0 - w[-1], abs=1e-12)


@pytest.mark.parametrize("n,frac,kind,seed", [
    (1024, 0.10, "uniform", 1), (1024, 0.30, "uniform", 2), (1500, 0.05, "uniform", 3),
    (2048, 0.20, "clustered", 3000), (2048, 0.05, "clustered", 3001), (1200, 0.50, "uniform", 4),
])
def test_slq_threshold_leaves_k_beyond_it(n, frac, kind, seed):
    """On constructed spectra the stochastic threshold has at least k eigenvalues of A' at or
    below it, and not many more (at most k + 10 % of n)."""
    p = I.eig_uniform(n, seed, frac) if kind == "uniform" else I.eig_clustered(n, seed, frac)
    lamp = np.sort(-p.lam)                # A' = -A: the largest of A are the smallest of A'
    t = O.threshold_from_count_eig_slq(p.A, -1.0, p.k, seed)
    assert t is not None
    cnt = int(np.count_nonzero(lamp <= t))
    assert p.k <= cnt <= p.k + 0.10 * n, (cnt, p.k)


def test_slq_probe_seeds_are_distinct():
    seeds = {slq_probe_seed(1234, j) for j in range(16)}
    assert len(seeds) == 16 and all(0 <= s < 2 ** 64 for s in seeds)


def test_partial_eig_with_slq_threshold():
    """n = 1024, 25 % largest (a wide block: the stochastic threshold is used) against the
    constructed spectrum at the FP64 tolerances."""
    p = I.eig_uniform(1024, 9, 0.25)
    r = O.qdwhp_eig(p.A, O.EigOptions(k=p.k))
    m = O.eig_metrics(p.A, r.lam, r.V, np.sort(p.lam)[::-1][: p.k])
    assert m["lam_err"] <= 1e-12 and m["orth"] <= 5e-15 * 1024 and m["resid"] <= 1e-13, m
    assert r.retries == 0
