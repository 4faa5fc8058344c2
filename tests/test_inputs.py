"""The seeded input generators (no method arithmetic): the Haar construction of the workloads and
the random butterfly construction of the serving stream, checked on the host (torch CPU): known
spectra reproduced to rounding, orthogonal factors, dense matrices, and the stream's recipe."""

import math

import numpy as np
import pytest

from paper_2104_14186_gb300 import inputs as I

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("n", [1, 2, 7, 200, 513])
def test_butterfly_eig_has_the_drawn_spectrum(n):
    A, lam, k = I.eig_butterfly_device(n, 3, 0.1, device="cpu")
    A = A.numpy()
    assert np.array_equal(A, A.T)
    ev = np.linalg.eigvalsh(A)
    assert np.max(np.abs(np.sort(lam) - ev)) <= 1e-14 * max(1, math.log2(n))
    assert k == I.k_from_fraction(n, 0.1)
    if n > 2:
        assert np.mean(np.abs(A) > 1e-14) > 0.99          # dense, not diagonal plus a few rotations


@pytest.mark.parametrize("m,n", [(1, 1), (300, 200), (513, 257), (400, 400)])
def test_butterfly_svd_has_the_drawn_singular_values(m, n):
    A, sigma, k = I.svd_butterfly_device(m, n, 4, 0.1, device="cpu")
    sv = np.linalg.svd(A.numpy(), compute_uv=False)
    assert A.shape == (m, n)
    assert np.max(np.abs(sigma - sv)) <= 1e-14 * max(1, math.log2(m))
    assert sigma[0] == 1.0 and (n == 1 or abs(sigma[-1] - 1e-10) < 1e-24)


def test_butterfly_factor_is_orthogonal_and_spread():
    """Four sweeps: orthogonal to rounding, and the largest entry near a Haar factor's."""
    for n in (256, 1000):
        g = torch.Generator().manual_seed(5)
        Qm = I._apply_rows(torch.eye(n, dtype=torch.float64), I._butterfly_layers(n, g, "cpu")).numpy()
        assert np.linalg.norm(Qm.T @ Qm - np.eye(n)) <= 1e-13
        assert np.abs(Qm).max() <= 1.3 * math.sqrt(2 * math.log(n) / n) * 1.2


def test_butterfly_inputs_are_seeded():
    a1 = I.eig_butterfly_device(64, 11, 0.2, device="cpu")[0]
    a2 = I.eig_butterfly_device(64, 11, 0.2, device="cpu")[0]
    a3 = I.eig_butterfly_device(64, 12, 0.2, device="cpu")[0]
    assert torch.equal(a1, a2) and not torch.equal(a1, a3)


def test_serving_stream_recipe():
    """2000 requests: about half EIG (n in [128, 8192]), half SVD (n in [128, 4096], m in
    [n, 2n]), fractions in [0.01, 0.20], unit-rate exponential gaps."""
    reqs, gaps = I.serving_stream(2000, 5000)
    eig = [r for r in reqs if r["kind"] == "eig"]
    svd = [r for r in reqs if r["kind"] == "svd"]
    assert len(reqs) == 2000 and 900 <= len(eig) <= 1100
    assert all(128 <= r["n"] <= 8192 and r["m"] == r["n"] for r in eig)
    assert all(128 <= r["n"] <= 4096 and r["n"] <= r["m"] <= 2 * r["n"] for r in svd)
    assert max(r["n"] for r in eig) > 7000 and max(r["n"] for r in svd) > 3500
    assert all(0.01 <= r["fraction"] <= 0.20 for r in reqs)
    assert gaps.shape == (2000,) and np.all(gaps > 0) and abs(gaps.mean() - 1.0) < 0.1
