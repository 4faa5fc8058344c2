"""The mixed-precision path (QDWHP_MIXED): every Cholesky-based QDWH step but the last in
FP32, everything else in FP64.  Its accuracy is stated per result:
  * without refinement, eigen/singular values are accurate to ~1e-6 (EIG) / ~1e-12 (SVD)
    relative to ||A||_2 but vectors only to ~1e-4 / ~1e-6: the FP32 rounding (u_32 = 6e-8)
    of the iterates, amplified by the condition of Z = I + c X^T X (up to ~1.5e3 when the
    unwanted side is scaled by the guard's limit of ~9), rotates the captured subspace;
  * with FP64 subspace-iteration steps on Q2 (refine_steps) the SVD reaches the FP64
    tolerances again."""

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


def test_mixed_eig_stated_accuracy(Q):
    p = I.eig_uniform(512, 1000, 0.10)
    r = Q.eig(dev(p.A), k=p.k, precision=Q.MIXED)
    assert r.info["it_f32"] == 2
    m = O.eig_metrics(p.A, r.lam.cpu().numpy(), r.V.cpu().numpy(), np.sort(p.lam)[::-1][: p.k])
    assert m["lam_err"] <= 1e-6, m
    assert m["resid"] <= 1e-3, m
    assert m["orth"] <= 5e-15 * 512, m


def test_mixed_svd_without_refinement_stated_accuracy(Q):
    q = I.svd_logspaced(1024, 1024, 2002, 0.05)
    r = Q.svd(dev(q.A), k=q.k, precision=Q.MIXED)
    assert r.info["it_f32"] >= 1
    m = O.svd_metrics(q.A, r.sigma.cpu().numpy(), r.U.cpu().numpy(), r.V.cpu().numpy(), q.sigma[: q.k])
    assert m["sigma_err"] <= 1e-10, m
    assert m["residU"] <= 1e-4 and m["residV"] <= 1e-13, m


def test_mixed_svd_refined_meets_fp64_tolerances_full_size(Q):
    """The SVD workload (4096 x 4096, top 5 %) in mixed precision with 6 FP64 refinement
    steps meets the plain-FP64 tolerances and agrees with the oracle."""
    q = I.svd_logspaced(4096, 4096, 2000, 0.05)
    r = Q.svd(dev(q.A), k=q.k, precision=Q.MIXED, refine_steps=6)
    assert r.info["it_f32"] == 2
    sig, U, V = r.sigma.cpu().numpy(), r.U.cpu().numpy(), r.V.cpu().numpy()
    m = O.svd_metrics(q.A, sig, U, V, q.sigma[: q.k])
    assert m["sigma_err"] <= 1e-12, m
    assert m["orthU"] <= 5e-15 * 4096 and m["orthV"] <= 5e-15 * 4096, m
    assert m["residV"] <= 1e-13 and m["residU"] <= 1e-13, m
