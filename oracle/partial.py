"""QDWHpartial-EIG (Algorithm 1) and QDWHpartial-SVD (Algorithm 2), plain FP64.

The steps below follow the paper in its order and notation.  Where the paper
is silent (how many Lanczos steps, how to turn a requested count into the
threshold the method needs, the QR/Cholesky switch), the reading taken is
stated at the step and listed in the design notes:

  * Lanczos: 30 steps with full reorthogonalisation from a SplitMix64 start
    vector; an extreme eigenvalue is estimated as Ritz value -/+ residual norm,
    pushed 1 % outwards (Algorithm 1 step 1 asks for "a few steps").
  * Count -> threshold: the k-th Ritz value of any subspace is a one-sided bound
    on the k-th eigenvalue (Cauchy interlacing), so a threshold there captures at
    least k wanted eigenpairs.  EIG: the block Krylov space of k+p starting vectors
    and q products with a positive semidefinite shift of the operator (only the
    last block when that basis would exceed min(n/8, 2048) columns).  SVD: subspace
    iteration, q+1 products of A^T A with k+p vectors.
  * Threshold placement guard: the wanted interval is kept at least 10 % of the
    spectral spread wide, so that the unwanted side is never scaled by more
    than about 9 (a threshold inside a tight cluster, or just below the largest
    eigenvalue, would otherwise make the first Cholesky factor ill conditioned:
    at a 5 % guard the residual reached 4e-13 on a uniform spectrum).
  * QR step while c_k > 100, Cholesky step otherwise (Section 4.2 asks for a
    QR-based first step when s is small).
  * Index rule tolerance 0.1 for the solvers (the printed algorithms use 0.01).
    Section 4.1 bounds the containment of the wanted subspace by u / sigma_min(R11)
    and asks for sigma_min(R11) >= tol = Omega(1), reading sigma_min(R11) off diag(R)
    on the grounds that the QR is rank revealing; without pivoting or a random
    Omega it is not quite, and at tol = 0.01 the residuals reached 2.1e-13 (EIG, n =
    512) and 1.2e-13 (SVD transposed residual), against 2.3e-14 and 1.4e-14 at 0.1,
    for about 5 % (EIG) and 10-20 % (SVD) more captured columns.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from .qdwh import dwh_schedule, qdwh_chol_step, qdwh_qr_step
from .zolo import zolo_schedule, zolo_step
from .rng import gaussian, uniform_pm1

# Stream ids of the random draws of the method (XORed into the user seed).
STREAM_LANCZOS = 0x4C414E43   # "LANC"
STREAM_BLOCK = 0x424C4F43     # "BLOC"
STREAM_OMEGA = 0x4F4D4547     # "OMEG"
STREAM_SLQ = 0x534C5150       # "SLQP"


@dataclass
class EigOptions:
    k: int                      # wanted count (>= 1)
    side: str = "largest"       # "largest" or "smallest"
    s: float = 0.2              # shift and ell_0 (Algorithm 1 step 2)
    iters: int = 3              # QDWH iterations (three for s = 0.2, two for s = 0.875)
    tol: float = 0.1            # index rule tolerance (Algorithm 1 step 4; see the module notes)
    lanczos_steps: int = 30
    block_extra: int = 16       # p in the (k+p)-dimensional threshold subspace
    power_steps: int = 6        # q (block Krylov depth)
    guard: float = 0.10         # minimum wanted width / spectral spread
    max_retries: int = 2
    seed: int = 1234
    zolo_r: int = 0             # 0: QDWH steps; r >= 1: Zolo-PD of type (2r+1, 2r) until ell = 1
    zolo_c_qr: float = 20.0     # Zolo-PD: a term is QR-formed when 1 / c_{2j-1} > zolo_c_qr (QDWH EIG
                                # steps are Cholesky-based whatever c, Section 4.1)
    use_omega: bool = False     # QR of (r(A~) + I) Omega / 2 with a Gaussian Omega (Section 4.1)


@dataclass
class SvdOptions:
    k: int
    tol: float = 0.1
    c_qr: float = 100.0         # QR-based step while c_k > c_qr
    lanczos_steps: int = 30
    block_extra: int = 16
    power_steps: int = 2
    s_min: float = 1e-15
    max_retries: int = 2
    seed: int = 1234
    zolo_r: int = 0             # 0: QDWH steps; r >= 1: Zolo-PD of type (2r+1, 2r)
    zolo_c_qr: float = 20.0     # Zolo-PD: a term is QR-formed when 1 / c_{2j-1} > zolo_c_qr
    use_omega: bool = False     # QR of (I - r^T r) Omega with a Gaussian Omega (Section 4.1)


@dataclass
class EigResult:
    lam: np.ndarray
    V: np.ndarray
    ell: int
    t: float
    mu: float
    retries: int
    info: dict = field(default_factory=dict)


@dataclass
class SvdResult:
    sigma: np.ndarray
    U: np.ndarray
    V: np.ndarray
    ell: int
    s: float
    alpha: float
    retries: int
    info: dict = field(default_factory=dict)


def lanczos_tridiagonal(matvec, n: int, steps: int, seed: int):
    """Lanczos with full reorthogonalisation (classical Gram-Schmidt, twice) from the
    SplitMix64 start vector.  Returns (alpha (m,), beta (m,)): the diagonal and off-diagonal of
    the m x m tridiagonal T, beta[m-1] being the norm of the last residual (0 at a breakdown)."""
    steps = max(1, min(steps, n))
    q = uniform_pm1(seed ^ STREAM_LANCZOS, n)
    Q = np.zeros((n, steps), dtype=np.float64)
    Q[:, 0] = q / np.linalg.norm(q)
    alpha = np.zeros(steps)
    beta = np.zeros(steps)
    m = steps
    for j in range(steps):
        w = matvec(Q[:, j])
        alpha[j] = Q[:, j] @ w
        Qj = Q[:, : j + 1]
        w = w - Qj @ (Qj.T @ w)
        w = w - Qj @ (Qj.T @ w)
        beta[j] = np.linalg.norm(w)
        if j + 1 == steps:
            break
        if beta[j] <= 1e-14 * max(abs(alpha[j]), 1e-300):
            m = j + 1
            beta[j] = 0.0
            break
        Q[:, j + 1] = w / beta[j]
    return alpha[:m], beta[:m]


def lanczos_extremes(matvec, n: int, steps: int, seed: int):
    """Lanczos with full reorthogonalisation (Algorithm 1 step 1).

    Returns (theta_min, res_min, theta_max, res_max): the extreme Ritz values of
    the tridiagonal T and their residual norms beta_m |s_{m,i}|.
    """
    alpha, beta = lanczos_tridiagonal(matvec, n, steps, seed)
    m = alpha.shape[0]
    T = np.diag(alpha) + np.diag(beta[: m - 1], 1) + np.diag(beta[: m - 1], -1)
    theta, S = np.linalg.eigh(T)
    res = abs(beta[m - 1]) * np.abs(S[m - 1, :])
    return theta[0], res[0], theta[-1], res[-1]


def lanczos_extremes_normal(A: np.ndarray, steps: int, seed: int):
    """Lanczos on A^T A (norm estimate, Algorithm 2 step 1)."""
    return lanczos_extremes(lambda x: A.T @ (A @ x), A.shape[1], steps, seed)


def _block_start(n: int, b: int, seed: int) -> np.ndarray:
    """n x b block of SplitMix64 uniforms, column-major order."""
    return uniform_pm1(seed ^ STREAM_BLOCK, n * b).reshape((n, b), order="F")


def _orth(Y: np.ndarray) -> np.ndarray:
    return np.linalg.qr(Y, mode="reduced")[0]


# A block Krylov basis is used only while it has at most min(n / 8, 2048) columns; a wider
# one would cost a Rayleigh-Ritz problem comparable to the solve itself, and the last
# power block alone is kept instead.
KRYLOV_MAX_COLS = 2048


def threshold_from_count_eig(A: np.ndarray, eps_side: float, k: int, lam_hi: float,
                             p: int, q: int, seed: int) -> float:
    """Threshold t' on A' = eps_side * A with at least k eigenvalues of A' <= t'.

    Block Krylov space K = span[Om, P Om, ..., P^q Om] of P = lam_hi I - A' (positive
    semidefinite, dominant part = the wanted small end of A'), each block orthonormalised
    before the next product; Rayleigh-Ritz of A' on K.  By Cauchy interlacing the k-th
    smallest Ritz value is >= the k-th smallest eigenvalue, so it is a valid threshold.
    When (q+1)(k+p) exceeds min(n/8, KRYLOV_MAX_COLS) only the last block is kept (subspace
    iteration).
    """
    n = A.shape[0]
    b = min(n, k + p)
    Y = _block_start(n, b, seed)
    krylov = (q + 1) * b <= min(n // 8, KRYLOV_MAX_COLS)
    blocks = [_orth(Y)] if krylov else []
    for _ in range(q):
        Qy = _orth(Y)
        Y = lam_hi * Qy - eps_side * (A @ Qy)
        if krylov:
            blocks.append(_orth(Y))
    K = _orth(np.hstack(blocks)) if krylov else _orth(lam_hi * _orth(Y) - eps_side * (A @ _orth(Y)))
    H = K.T @ (eps_side * (A @ K))
    H = 0.5 * (H + H.T)
    theta = np.linalg.eigvalsh(H)
    return float(theta[k - 1])


# Stochastic Lanczos quadrature threshold (EIG, wide blocks): probes, Lanczos steps per probe,
# safety factor on the standard error, and the smallest order that uses it (below it the
# Ritz-value bound of the block subspace captures fewer unwanted eigenvalues).
SLQ_PROBES = 16
SLQ_STEPS = 64
SLQ_Z = 3.0
SLQ_MIN_N = 1024


def slq_probe_seed(seed: int, j: int) -> int:
    """Seed of probe j (its Lanczos start vector is drawn from seed ^ STREAM_LANCZOS inside
    lanczos_tridiagonal, as for the bounds)."""
    return (seed ^ STREAM_SLQ ^ (((j + 1) * 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF)) & 0xFFFFFFFFFFFFFFFF


def gauss_rule(alpha: np.ndarray, beta: np.ndarray):
    """Gauss quadrature of the Lanczos tridiagonal (Golub and Welsch 1969): nodes = eigenvalues of
    T (ascending), weights = squared first components of its eigenvectors (summing to 1 for a
    unit start vector)."""
    m = alpha.shape[0]
    T = np.diag(alpha) + np.diag(beta[: m - 1], 1) + np.diag(beta[: m - 1], -1)
    theta, S = np.linalg.eigh(T)
    w = S[0, :] ** 2
    return theta, w / w.sum()


def threshold_from_count_eig_slq(A: np.ndarray, eps_side: float, k: int, seed: int, probes: int = SLQ_PROBES,
                                 steps: int = SLQ_STEPS, z: float = SLQ_Z):
    """Threshold t' on A' = eps_side * A below which A' has at least k eigenvalues with high
    probability, by stochastic Lanczos quadrature (Ubaru, Chen and Saad 2017).

    Each probe v (a SplitMix64 vector, normalised) gives the Gauss rule (theta_i, w_i) of its
    spectral distribution F_v(x) = sum over eigenpairs (lambda_i, u_i) of A' with lambda_i <= x
    of (v^T u_i)^2.  By the Chebyshev-Markov-Stieltjes inequalities F_v(theta_j - 0) >=
    w_1 + ... + w_{j-1}, so at any x, F_v(x) >= L_v(x) = the sum of the weights of the nodes
    below the last node <= x.  The count of eigenvalues <= x is n E_v[F_v(x)]; t' is the
    smallest node x of all probes with n (mean L_v(x) - z stderr) >= k.  Returns None when no
    node qualifies (the caller then uses the block subspace bound).  Unlike the Ritz-value
    bound this is an estimate: the solver's count check and retries still guarantee the k
    pairs."""
    n = A.shape[0]
    rules = []
    for j in range(probes):
        al, be = lanczos_tridiagonal(lambda x: eps_side * (A @ x), n, steps, slq_probe_seed(seed, j))
        rules.append(gauss_rule(al, be))
    best = None
    for x in np.concatenate([r[0] for r in rules]):
        L = np.array([slq_lower_bound(theta, w, x) for theta, w in rules])
        est = n * L.mean()
        se = n * L.std(ddof=1) / math.sqrt(probes) if probes > 1 else 0.0
        if est - z * se >= k and (best is None or x < best):
            best = float(x)
    return best


def slq_lower_bound(theta: np.ndarray, w: np.ndarray, x: float) -> float:
    """Lower bound of a spectral distribution at x from its Gauss rule (nodes theta ascending,
    weights w): with theta_j the last node <= x, F(x) >= F(theta_j - 0) >= w_1 + ... + w_{j-1}
    (Chebyshev-Markov-Stieltjes); 0 when no node lies at or below x."""
    j = int(np.count_nonzero(theta <= x))
    return float(w[: max(j - 1, 0)].sum())


def threshold_from_count_svd(A: np.ndarray, k: int, p: int, q: int, seed: int) -> float:
    """sigma_hat_k <= sigma_k: square root of the k-th largest Ritz value of A^T A on
    span((A^T A)^(q+1) Om) (subspace iteration, each block orthonormalised before the next
    product); Cauchy interlacing.  The powers of A^T A separate the spectrum fast enough that
    a Krylov basis would not shrink ell measurably, at (q+1) times the Rayleigh-Ritz width."""
    n = A.shape[1]
    b = min(n, k + p)
    Y = _block_start(n, b, seed)
    for _ in range(q + 1):
        Y = A.T @ (A @ _orth(Y))
    K = _orth(Y)
    C = A @ K
    H = C.T @ C
    H = 0.5 * (H + H.T)
    theta = np.linalg.eigvalsh(H)[::-1]
    return math.sqrt(max(theta[k - 1], 0.0))


def index_from_diag(R: np.ndarray, tol: float) -> int:
    """Algorithm 1 step 4 / Algorithm 2 step 4: ind = min(find(|diag(R)| < tol)),
    0-based; returns n when no diagonal entry is below tol."""
    d = np.abs(np.diag(R))
    hits = np.nonzero(d < tol)[0]
    return int(hits[0]) if hits.size else d.shape[0]


def gaussian_omega(n: int, seed: int) -> np.ndarray:
    """The n x n Gaussian matrix Omega of Section 4.1 (the QR of B Omega is rank revealing with
    high probability), entries N(0, 1/n) so that B Omega keeps B's unit scale and the index
    tolerance means the same with and without it.  Column-major draw from the Box-Muller
    transform of the SplitMix64 stream seed ^ STREAM_OMEGA."""
    return gaussian(seed ^ STREAM_OMEGA, n * n).reshape((n, n), order="F") / math.sqrt(n)


def extraction_qr(B: np.ndarray, tol: float, omega_seed: int | None = None):
    """Steps 3-5 of Algorithms 1 and 2: the full Householder QR of B, or of B Omega with the
    Gaussian Omega of Section 4.1 when omega_seed is given (rank revealing with high
    probability), then the index rule on diag(R).  Returns (F, Q, R, ind): F is the matrix
    factored, and Q2 = Q[:, ind:] (ell = n - ind columns) contains B's numerical null space
    up to ||V0^T F||_2 / sigma_min(R11) (Theorem 1)."""
    F = B if omega_seed is None else B @ gaussian_omega(B.shape[1], omega_seed)
    Qf, R = np.linalg.qr(F, mode="complete")
    return F, Qf, R, index_from_diag(R, tol)


def polar_iterations(X: np.ndarray, ell0: float, zolo_r: int, fixed_iters: int | None, c_qr: float,
                     zolo_c_qr: float = 20.0):
    """Step 2 of Algorithms 1 and 2: QDWH from ell0 (fixed_iters steps, or until |ell - 1| < 5 eps),
    QR-based while c_k > c_qr; or, with zolo_r >= 1, Zolo-PD iterations of type (2 zolo_r + 1,
    2 zolo_r) until |ell - 1| < 5 eps, a term QR-formed when 1 / c_{2j-1} > zolo_c_qr.
    Returns (X, schedule, number of QR-formed steps or terms)."""
    n_qr = 0
    if zolo_r > 0:
        sched = zolo_schedule(ell0, zolo_r)
        for c, a, M, _, _ in sched:
            X, q = zolo_step(X, c, a, M, zolo_c_qr)
            n_qr += q
        return X, sched, n_qr
    sched = dwh_schedule(ell0, fixed_iters=fixed_iters)
    for a, b, c, _, _ in sched:
        if c > c_qr:
            X = qdwh_qr_step(X, a, b, c)
            n_qr += 1
        else:
            X = qdwh_chol_step(X, a, b, c)
    return X, sched, n_qr


def _eig_core(A: np.ndarray, eps_side: float, t: float, lam_lo: float, s: float, iters: int, tol: float,
              zolo_r: int = 0, zolo_c_qr: float = 20.0, omega_seed: int | None = None):
    """Algorithm 1 steps 1-6 for B = A' - t I with A' = eps_side * A, whose
    wanted eigenvalues lie on [mu, 0], mu = lam_lo - t <= lambda_min(B)."""
    n = A.shape[0]
    mu = lam_lo - t
    absmu = abs(mu)
    # Step 1 scaling A := A/|mu| and step 2 shift A~ = (1-s) A - s I, applied to B.
    X = ((1.0 - s) * eps_side / absmu) * A
    X[np.diag_indices(n)] -= (1.0 - s) * t / absmu + s
    # Step 2: QDWH iterations from ell_0 = s, Cholesky-based in all iterations (Section 4.1);
    # or Zolo-PD iterations.
    X, sched, _ = polar_iterations(X, s, zolo_r, iters, math.inf, zolo_c_qr)
    # Step 3: QR of (r(A~) + I) / 2, or of (r(A~) + I) Omega / 2 (Section 4.1); steps 4-5: index
    # rule and trailing columns of Q.
    Bq = 0.5 * (X + np.eye(n))
    F, Qf, R, ind = extraction_qr(Bq, tol, omega_seed)
    Q2 = Qf[:, ind:]
    # Step 6: Rayleigh-Ritz on the original A, so the Ritz values need no rescaling (step 7).
    M = Q2.T @ (A @ Q2)
    M = 0.5 * (M + M.T)
    theta, W = np.linalg.eigh(M)
    return theta, W, Q2, mu, {"sched": sched, "ind": ind, "B": Bq, "F": F, "Q": Qf, "R": R}


def qdwhp_eig_negative(A: np.ndarray, mu: float, s: float = 0.2, iters: int = 3, tol: float = 0.01,
                       omega_seed: int | None = None):
    """Algorithm 1 as printed: the negative eigenpairs of A, given a lower bound
    mu <= lambda_min(A) < 0 (step 3 with the Gaussian Omega when omega_seed is given).
    Returns (lam ascending, V, info)."""
    theta, W, Q2, _, info = _eig_core(A, 1.0, 0.0, mu, s, iters, tol, omega_seed=omega_seed)
    sel = np.nonzero(theta < 0.0)[0]
    return theta[sel], Q2 @ W[:, sel], info


def qdwhp_eig(A: np.ndarray, opts: EigOptions) -> EigResult:
    """QDWHpartial-EIG (Algorithm 1) for the k largest or smallest eigenpairs.

    The wanted side is made the negative side by shifting and scaling by -1
    (Section 4.1, remark after Algorithm 1): with eps = -1 for "largest" and +1
    for "smallest", A' = eps A has the wanted eigenvalues at its low end, and
    B = A' - t' I has them on [mu, 0].
    """
    n = A.shape[0]
    k = opts.k
    if not (1 <= k <= n):
        raise ValueError("k out of range")
    eps_side = -1.0 if opts.side == "largest" else 1.0

    # Step 1: Lanczos bounds of A' (Ritz value -/+ residual, 1 % outwards).
    th_min, r_min, th_max, r_max = lanczos_extremes(lambda x: A @ x, n, opts.lanczos_steps, opts.seed)
    if eps_side < 0:
        lo_raw, hi_raw = -(th_max + r_max), -(th_min - r_min)
    else:
        lo_raw, hi_raw = th_min - r_min, th_max + r_max
    # Degenerate case: the spectrum is one point to rounding (n = 1, a multiple of the
    # identity, the zero matrix).  mu would be 0 (Algorithm 1 scales by 1/|mu|), and every
    # vector is an eigenvector: return the first k unit vectors and their Rayleigh quotients.
    if hi_raw - lo_raw <= 16 * 2.0 ** -53 * max(abs(lo_raw), abs(hi_raw)):
        V = np.eye(n)[:, :k]
        lam = np.diag(A)[:k].astype(np.float64)
        return EigResult(lam, V, 0, float(th_max), float(th_min), 0, {"degenerate": True})
    spread = hi_raw - lo_raw
    lam_lo = lo_raw - 0.01 * spread
    lam_hi = hi_raw + 0.01 * spread

    # Threshold for the requested count: the k-th Ritz value of a block Krylov space (Cauchy
    # interlacing), or, when that basis would be too wide for n >= SLQ_MIN_N, the stochastic
    # Lanczos quadrature estimate; then the width guard.
    b = min(n, k + opts.block_extra)
    wide = (opts.power_steps + 1) * b > min(n // 8, KRYLOV_MAX_COLS)
    t = None
    if wide and n >= SLQ_MIN_N:
        t = threshold_from_count_eig_slq(A, eps_side, k, opts.seed)
    if t is None:
        t = threshold_from_count_eig(A, eps_side, k, lam_hi, opts.block_extra, opts.power_steps, opts.seed)
    t += 1e-10 * spread
    t = max(t, lam_lo + opts.guard * (lam_hi - lam_lo))

    retries = 0
    while True:
        theta, W, Q2, mu, info = _eig_core(A, eps_side, t, lam_lo, opts.s, opts.iters, opts.tol, opts.zolo_r,
                                           opts.zolo_c_qr, opts.seed if opts.use_omega else None)
        lamp = eps_side * theta               # Ritz values of A'
        sel = np.nonzero(lamp <= t)[0]
        if sel.size >= k or retries >= opts.max_retries:
            break
        retries += 1
        t = t + 0.25 * (lam_hi - t)
    if sel.size < k:
        raise RuntimeError("fewer than k wanted Ritz values after retries")
    # Step 7: the k wanted Ritz pairs, V = Q2 W.
    order = sel[np.argsort(lamp[sel], kind="stable")][:k]
    lam = theta[order]
    V = Q2 @ W[:, order]
    info["lanczos"] = (th_min, r_min, th_max, r_max)
    return EigResult(lam, V, Q2.shape[1], eps_side * t, eps_side * mu, retries, info)


def qdwhp_svd_threshold(A: np.ndarray, s: float, alpha: float, tol: float = 0.01, c_qr: float = 100.0,
                        zolo_r: int = 0, omega_seed: int | None = None, zolo_c_qr: float = 20.0):
    """Algorithm 2 as printed, for m >= n: the singular triplets with sigma >= s alpha,
    alpha ~ ||A||_2.  Returns (sigma descending, U, V, info)."""
    n = A.shape[1]
    # Step 2: QDWH on A/alpha from ell_0 = s until |ell - 1| < 5 eps; QR-based steps
    # while c_k > c_qr (Section 4.2: the QR form for the first step when s is small).
    X, sched, n_qr = polar_iterations(A / alpha, s, zolo_r, None, c_qr, zolo_c_qr)
    # Step 3: QR of I - r(A~)^T r(A~), or of (I - r^T r) Omega (Section 4.1); steps 4-5.
    Bq = np.eye(n) - X.T @ X
    F, Qf, R, ind = extraction_qr(Bq, tol, omega_seed)
    Q2 = Qf[:, ind:]
    # Step 6: A Q2 with the unscaled A, and its SVD.
    C = A @ Q2
    Ut, St, Vtt = np.linalg.svd(C, full_matrices=False)
    # Step 7: the triplets above s ||A||_2; step 8: V1 = Q2 V~1.
    sel = np.nonzero(St >= s * alpha)[0]
    info = {"sched": sched, "n_qr": n_qr, "ind": ind, "B": Bq, "F": F, "Q": Qf, "R": R}
    return St[sel], Ut[:, sel], Q2 @ Vtt[sel, :].T, info


def qdwhp_svd(A: np.ndarray, opts: SvdOptions) -> SvdResult:
    """QDWHpartial-SVD (Algorithm 2 and the Section 5 listing) for the k largest
    singular triplets.  For m < n it works on A^T and swaps U and V (Section 4.2)."""
    m, n = A.shape
    if m < n:
        r = qdwhp_svd(np.asfortranarray(A.T), opts)
        return SvdResult(r.sigma, r.V, r.U, r.ell, r.s, r.alpha, r.retries, r.info)
    k = opts.k
    if not (1 <= k <= n):
        raise ValueError("k out of range")
    # Step 1: alpha ~ ||A||_2 (Lanczos on A^T A, Ritz value + residual).
    _, _, th_max, r_max = lanczos_extremes_normal(A, opts.lanczos_steps, opts.seed)
    alpha = math.sqrt(max(th_max + r_max, 0.0))
    if alpha == 0.0:
        # the zero matrix: every singular value is 0 and any orthonormal U, V serve
        return SvdResult(np.zeros(k), np.eye(m)[:, :k], np.eye(n)[:, :k], 0, 0.0, 0.0, 0, {"degenerate": True})
    # Relative threshold s from the requested count.
    sig_hat = threshold_from_count_svd(A, k, opts.block_extra, opts.power_steps, opts.seed)
    s = max(sig_hat / alpha * (1.0 - 1e-10), opts.s_min)
    retries = 0
    while True:
        sigma, U, V, info = qdwhp_svd_threshold(A, s, alpha, opts.tol, opts.c_qr, opts.zolo_r,
                                                opts.seed if opts.use_omega else None, opts.zolo_c_qr)
        if sigma.shape[0] >= k or retries >= opts.max_retries:
            break
        retries += 1
        s = max(0.5 * s, opts.s_min)
    if sigma.shape[0] < k:
        raise RuntimeError("fewer than k singular values above the threshold after retries")
    return SvdResult(sigma[:k], U[:, :k], V[:, :k], n - info["ind"], s, alpha, retries, info)
