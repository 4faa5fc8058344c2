"""Plain FP64 CPU oracle for QDWHpartial-EIG and QDWHpartial-SVD.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code with the CUDA library; both sides take
their inputs from ``paper_2104_14186_gb300.inputs`` and each implements the
SplitMix64 counter generator for the random vectors the method draws.

The oracle follows the paper step by step (Algorithm 1 for EIG, Algorithm 2
and the ScaLAPACK listing of Section 5 for SVD), with numpy/LAPACK routines
(matmul, Householder QR, Cholesky, triangular solve, dense symmetric
eigensolver, dense SVD) as the individual steps.  Every public function names
the passage it follows.

Parity status per function (what pins it, see tests/test_oracle_*.py):
  dwh_weights            pinned: closed-form optimality of the (3,2) function,
                         iteration counts printed in the paper
  qdwh_chol_step         pinned: spectral-map identity on known spectra
  qdwh_qr_step           pinned: spectral-map identity; equals the Cholesky step
  qdwh_polar             pinned: polar factor from the SVD, H symmetric PSD
  lanczos_extremes       pinned: bounds against the known spectrum
  threshold_from_count   pinned: Cauchy interlacing (k eigenvalues beyond t)
  gauss_rule / slq_*     pinned: the Gauss rule integrates polynomials of degree <= 2m - 1
                         exactly; its lower bound never exceeds the exact spectral
                         distribution (Chebyshev-Markov-Stieltjes) on known spectra; the
                         stochastic threshold leaves >= k eigenvalues beyond it on
                         constructed spectra
  qdwhp_eig / qdwhp_svd  pinned: constructed spectra, brute-force Jacobi (n<=64),
                         LAPACK eigh/svd, Theorem 1 containment bound
  extraction_qr          pinned: Theorem 1 containment bound with and without Omega; on a
                         Kahan matrix (unpivoted diag(R) far above sigma_min) only the
                         Omega form captures the null vector and its diag(R) tracks
                         sigma_min(R11)
  gaussian               pinned: Kolmogorov-Smirnov against the normal distribution,
                         moments, independence of the Box-Muller pair
  subspace size ell      parity unpinned (several ell are correct; only final
                         outputs are compared)
  syev                   the definition (all eigenpairs); pinned: constructed
                         spectra, brute-force Jacobi
  full.split / qdwh_eig  pinned: rank(C) = #eigenvalues above sigma, C = V+ V+^T
                         on known spectra; all eigenpairs against constructed spectra
  full.gesvd             the definition (all singular triplets); pinned: constructed
                         singular values, residuals, the eigenvalues of A^T A
  zolo.*                 pinned: r = 1 equals the QDWH weights, Chebyshev alternation
                         (2r + 2 points), composition law, spectral-map identity of both
                         term forms, polar factor from the SVD, iteration counts
  full.quadrature_median pinned: Gauss quadrature exact to degree 2m - 1, balance on a
                         12-decade spectrum, interior point of a two-point spectrum; the
                         unresolved-split measure trace(C) - ||C||_F^2 on a split at a
                         30-fold eigenvalue
  full.qdwh_svd          pinned: constructed singular values (to 1e-12 relative decades),
                         m < n, rank-deficient and zero matrices, residual invariants
"""

from .rng import splitmix64, uniform_pm1, gaussian  # noqa: F401
from .qdwh import dwh_weights, dwh_schedule, qdwh_chol_step, qdwh_qr_step, qdwh_polar, rational_map  # noqa: F401
from .partial import (  # noqa: F401
    EigOptions, SvdOptions, EigResult, SvdResult,
    lanczos_extremes, lanczos_extremes_normal, threshold_from_count_eig, threshold_from_count_svd,
    qdwhp_eig, qdwhp_svd, qdwhp_eig_negative, qdwhp_svd_threshold, index_from_diag, extraction_qr,
    gaussian_omega, threshold_from_count_eig_slq, gauss_rule, slq_lower_bound, lanczos_tridiagonal,
)
from .jacobi import jacobi_eig  # noqa: F401
from .full import syev  # noqa: F401
from . import full  # noqa: F401
from . import zolo  # noqa: F401
from .metrics import eig_metrics, svd_metrics  # noqa: F401
