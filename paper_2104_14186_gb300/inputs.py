"""Seeded synthetic test matrices with known spectra.

These generators build the inputs that the solver, its tests and the benchmark
share.  They hold none of the solver's arithmetic: each matrix is assembled as
``Q1 diag(d) Q2^T`` from Haar-distributed orthogonal factors, the construction
the paper's experiments use (Section 7.2: matrices from PDLATMS, mode 0, with
orthogonal factors taken from the QR factorization of random matrices; Q1 = Q2
for the symmetric case).  The spectra follow the workload definitions below.

Every draw comes from ``numpy.random.default_rng(seed)`` (PCG64), so a seed
fixes the matrix on every machine.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def haar_orthogonal(n: int, rng: np.random.Generator, m: int | None = None) -> np.ndarray:
    """m x n matrix with orthonormal columns, Haar distributed.

    Householder QR of an m x n N(0,1) matrix, with the columns of Q multiplied by
    sign(diag(R)) so that the distribution is exactly Haar (Mezzadri 2007).
    """
    m = n if m is None else m
    G = rng.standard_normal((m, n))
    Q, R = np.linalg.qr(G)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return np.asfortranarray(Q * d[None, :])


def symmetric_with_spectrum(lam: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    """A = Q diag(lam) Q^T with Haar Q, symmetrised exactly."""
    n = lam.shape[0]
    Q = haar_orthogonal(n, rng)
    A = (Q * lam[None, :]) @ Q.T
    A = 0.5 * (A + A.T)
    return np.asfortranarray(A)


def general_with_singular_values(m: int, sigma: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    """A = U diag(sigma) V^T, U m x n and V n x n Haar, m >= n = len(sigma)."""
    n = sigma.shape[0]
    U = haar_orthogonal(n, rng, m)
    V = haar_orthogonal(n, rng)
    return np.asfortranarray((U * sigma[None, :]) @ V.T)


@dataclass
class EigProblem:
    A: np.ndarray          # n x n symmetric, column-major
    lam: np.ndarray        # exact eigenvalues (unsorted, as drawn)
    k: int                 # wanted count
    side: str              # "largest" or "smallest"


@dataclass
class SvdProblem:
    A: np.ndarray          # m x n, column-major
    sigma: np.ndarray      # exact singular values, descending
    k: int


def k_from_fraction(n: int, fraction: float) -> int:
    """k = ceil(fraction * n), clamped to [1, n] (the library uses the same rule)."""
    k = int(math.ceil(fraction * n - 1e-9))
    return max(1, min(n, k))


def eig_uniform(n: int, seed: int, fraction: float = 0.10, side: str = "largest") -> EigProblem:
    """Symmetric n x n, eigenvalues uniform in [-1, 1] (EIG workload, n = 512, 10 % largest)."""
    rng = np.random.default_rng(seed)
    lam = rng.uniform(-1.0, 1.0, n)
    A = symmetric_with_spectrum(lam, rng)
    return EigProblem(A, lam, k_from_fraction(n, fraction), side)


def eig_clustered(n: int, seed: int, fraction: float, cluster_frac: float = 0.02) -> EigProblem:
    """Symmetric n x n: cluster_frac of the eigenvalues uniform in 1 +- 1e-6, the rest
    uniform in [-1, 0.9] (EIG workload n = 16384 with a tight cluster at the top)."""
    rng = np.random.default_rng(seed)
    nc = int(round(cluster_frac * n))
    lam = np.concatenate([rng.uniform(1.0 - 1e-6, 1.0 + 1e-6, nc), rng.uniform(-1.0, 0.9, n - nc)])
    A = symmetric_with_spectrum(lam, rng)
    return EigProblem(A, lam, k_from_fraction(n, fraction), "largest")


def svd_logspaced(m: int, n: int, seed: int, fraction: float = 0.05, decades: float = 12.0) -> SvdProblem:
    """m x n with sigma_i = 10^(-decades * i / (n - 1)), i = 0..n-1 (SVD workload:
    4096 x 4096, singular values log-spaced from 1 to 1e-12, top 5 %)."""
    rng = np.random.default_rng(seed)
    i = np.arange(n, dtype=np.float64)
    sigma = 10.0 ** (-decades * i / max(n - 1, 1))
    A = general_with_singular_values(m, sigma, rng)
    return SvdProblem(A, sigma, k_from_fraction(n, fraction))


def svd_geometric_half(n: int, seed: int) -> SvdProblem:
    """The paper's SVD test spectrum (Section 7.2): D[i] = 0.5^(100 i / n)."""
    rng = np.random.default_rng(seed)
    i = np.arange(n, dtype=np.float64)
    sigma = 0.5 ** (100.0 * i / n)
    A = general_with_singular_values(n, sigma, rng)
    return SvdProblem(A, sigma, 1)


def batch_sizes(count: int, seed: int, lo: int = 64, hi: int = 1024) -> np.ndarray:
    """Sizes of the batched workload: `count` sizes drawn uniformly from [lo, hi]."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=count)


def eig_clustered_device(n: int, seed: int, fraction: float, cluster_frac: float = 0.02, device="cuda"):
    """The clustered EIG workload built on the GPU (for sizes where a host QR of an n x n
    Gaussian matrix is too slow): same spectrum recipe as `eig_clustered`, with the
    Gaussian matrix drawn by torch's CUDA generator (Philox) from `seed` and its
    Householder QR done by torch.  Returns (A as a CUDA float64 tensor, lam as numpy, k)."""
    import torch

    rng = np.random.default_rng(seed)
    nc = int(round(cluster_frac * n))
    lam = np.concatenate([rng.uniform(1.0 - 1e-6, 1.0 + 1e-6, nc), rng.uniform(-1.0, 0.9, n - nc)])
    g = torch.Generator(device=device).manual_seed(seed)
    G = torch.randn(n, n, dtype=torch.float64, device=device, generator=g)
    Q, R = torch.linalg.qr(G)
    del G
    d = torch.sign(torch.diagonal(R))
    d[d == 0] = 1.0
    Q = Q * d[None, :]
    del R
    lam_t = torch.from_numpy(lam).to(device)
    A = (Q * lam_t[None, :]) @ Q.T
    A = 0.5 * (A + A.T)
    return A.contiguous(), lam, k_from_fraction(n, fraction)


def _haar_device(n: int, g, device, m: int | None = None):
    import torch
    m = n if m is None else m
    G = torch.randn(m, n, dtype=torch.float64, device=device, generator=g)
    Q, R = torch.linalg.qr(G)
    d = torch.sign(torch.diagonal(R))
    d[d == 0] = 1.0
    return Q * d[None, :]


def eig_uniform_device(n: int, seed: int, fraction: float = 0.10, device="cuda"):
    """`eig_uniform`'s spectrum (lambda ~ U[-1, 1] from numpy PCG64) with the Haar factor
    drawn and orthogonalised on the GPU (torch Philox generator + Householder QR).
    Returns (A as a CUDA float64 tensor, lam, k)."""
    import torch
    rng = np.random.default_rng(seed)
    lam = rng.uniform(-1.0, 1.0, n)
    g = torch.Generator(device=device).manual_seed(seed)
    Q = _haar_device(n, g, device)
    A = (Q * torch.from_numpy(lam).to(device)[None, :]) @ Q.T
    return (0.5 * (A + A.T)).contiguous(), lam, k_from_fraction(n, fraction)


def svd_logspaced_device(m: int, n: int, seed: int, fraction: float, decades: float = 10.0, device="cuda"):
    """`svd_logspaced`'s spectrum with Haar factors drawn on the GPU; returns (A, sigma, k)."""
    import torch
    i = np.arange(n, dtype=np.float64)
    sigma = 10.0 ** (-decades * i / max(n - 1, 1))
    g = torch.Generator(device=device).manual_seed(seed)
    U = _haar_device(n, g, device, m)
    V = _haar_device(n, g, device)
    A = (U * torch.from_numpy(sigma).to(device)[None, :]) @ V.T
    return A.contiguous(), sigma, k_from_fraction(n, fraction)


def _butterfly_layers(n: int, g, device, passes: int = 4):
    """Random orthogonal factor as a product of plane rotations (harness only): `passes` sweeps of
    butterfly layers with strides 1, 2, 4, ... < n, each rotating every pair (i, i + stride) with
    i's stride bit clear by a uniform random angle, and a random permutation before every sweep.
    Every coordinate mixes with every other within a sweep; after four sweeps the largest entry
    is within ~10 % of a Haar factor's typical largest entry (0.167 against 0.153 at n = 1000).
    The product is orthogonal to rounding (about 4 log2(n) u), and applying it costs
    O(n^2 log n) instead of a QR of an n x n Gaussian matrix.  Returns the operations in order: ("perm", p) or ("rot", i, j, c, s)."""
    import torch
    ops = []
    idx = torch.arange(n, device=device)
    for _ in range(passes):
        ops.append(("perm", torch.randperm(n, generator=g, device=device)))
        stride = 1
        while stride < n:
            i = idx[((idx // stride) % 2 == 0) & (idx + stride < n)]
            j = i + stride
            theta = torch.rand(i.numel(), generator=g, device=device, dtype=torch.float64) * (2 * math.pi)
            ops.append(("rot", i, j, torch.cos(theta), torch.sin(theta)))
            stride *= 2
    return ops


def _apply_rows(A, ops):
    """A := Q A for the orthogonal factor Q given by _butterfly_layers (in place on rows)."""
    for op in ops:
        if op[0] == "perm":
            A.copy_(A[op[1]])
        else:
            _, i, j, c, s = op
            Ai, Aj = A[i], A[j]
            A[i], A[j] = c[:, None] * Ai - s[:, None] * Aj, s[:, None] * Ai + c[:, None] * Aj
    return A


def eig_butterfly_device(n: int, seed: int, fraction: float, device="cuda"):
    """Symmetric n x n A = Q diag(lambda) Q^T with lambda ~ U[-1, 1] (numpy PCG64) and Q the random
    butterfly factor of _butterfly_layers (torch Philox from `seed`), built two-sided on the GPU in
    O(n^2 log n).  For the serving stream, whose 2000 inputs up to n = 8192 would take minutes of
    Householder QR to draw as Haar factors.  Returns (A as a CUDA float64 tensor, lam, k)."""
    import torch
    rng = np.random.default_rng(seed)
    lam = rng.uniform(-1.0, 1.0, n)
    g = torch.Generator(device=device).manual_seed(seed)
    ops = _butterfly_layers(n, g, device)
    A = torch.diag(torch.from_numpy(lam).to(device))
    _apply_rows(A, ops)
    At = A.t().contiguous()
    _apply_rows(At, ops)            # (Q (Q Lambda)^T)^T = Q Lambda Q^T
    A = 0.5 * (At + At.t())
    return A.contiguous(), lam, k_from_fraction(n, fraction)


def svd_butterfly_device(m: int, n: int, seed: int, fraction: float, decades: float = 10.0, device="cuda"):
    """m x n A = U [diag(sigma); 0] V^T (m >= n), sigma log-spaced over `decades` from 1, U and V
    random butterfly factors (as eig_butterfly_device).  Returns (A, sigma, k)."""
    import torch
    i = np.arange(n, dtype=np.float64)
    sigma = 10.0 ** (-decades * i / max(n - 1, 1))
    g = torch.Generator(device=device).manual_seed(seed)
    ops_u = _butterfly_layers(m, g, device)
    ops_v = _butterfly_layers(n, g, device)
    A = torch.zeros(m, n, dtype=torch.float64, device=device)
    A[torch.arange(n, device=device), torch.arange(n, device=device)] = torch.from_numpy(sigma).to(device)
    _apply_rows(A, ops_u)           # U [S; 0]
    At = A.t().contiguous()
    _apply_rows(At, ops_v)          # V (U [S; 0])^T = (U [S; 0] V^T)^T
    return At.t().contiguous(), sigma, k_from_fraction(n, fraction)


def serving_stream(count: int, seed: int, eig_n=(128, 8192), svd_n=(128, 4096), frac=(0.01, 0.20)):
    """Seeded request stream: half EIG (n uniform in eig_n, largest side), half SVD (n uniform in
    svd_n, m uniform in [n, 2n]); wanted fraction uniform in frac; unit-rate exponential
    inter-arrival gaps (scaled by the caller to the target rate)."""
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        f = float(rng.uniform(*frac))
        if rng.uniform() < 0.5:
            n = int(rng.integers(eig_n[0], eig_n[1] + 1))
            reqs.append({"kind": "eig", "m": n, "n": n, "fraction": f, "seed": seed * 100003 + i})
        else:
            n = int(rng.integers(svd_n[0], svd_n[1] + 1))
            m = int(rng.integers(n, 2 * n + 1))
            reqs.append({"kind": "svd", "m": m, "n": n, "fraction": f, "seed": seed * 100003 + i})
    gaps = rng.exponential(1.0, count)
    return reqs, gaps
