"""GPU parity of Zolo-PD (the type (2r+1, 2r) Zolotarev variant of QDWH, Section 3.1) in
both partial solvers, through the C ABI: the device schedule (Jacobi elliptic functions by
the AGM method) against the oracle's (scipy's elliptic functions), and the solutions
against the constructed spectra at the plain-FP64 tolerances."""

import numpy as np
import pytest

import oracle as O
from oracle import zolo as Z
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


def check_schedule(info, ell0, r):
    """The device's ell_k (Landen-transformation elliptic functions, accurate to a few ulps)
    against the oracle's (scipy's, whose relative error grows to ~1e-11 at ell = 1e-3 as the
    parameter 1 - ell^2 nears 1): agreement to 1e-10."""
    sched = Z.zolo_schedule(ell0, r)
    assert info["zolo_steps"] == len(sched), (info, len(sched))
    ref = np.array([s[4] for s in sched])
    got = np.array(info["ell_k"])
    assert np.all(np.abs(got - ref) <= 1e-10 * ref), (got, ref)
    assert abs(got[-1] - 1.0) < 5 * 2.0 ** -52


@pytest.mark.parametrize("r", [1, 2, 3])
@pytest.mark.parametrize("side", ["largest", "smallest"])
def test_eig_zolo(Q, r, side):
    """n = 512, 10 %: r = 1 reproduces QDWH's three steps, r = 2, 3 take two; at r = 2 and 3
    the first iteration's first shift is small enough (1 / c_1 > zolo_c_qr = 20) for the QR
    form, every other term is Cholesky-formed."""
    p = I.eig_uniform(512, 1000 + r, 0.10, side)
    res = Q.eig(dev(p.A), k=p.k, side=side, zolo_r=r)
    true = np.sort(p.lam)[::-1][: p.k] if side == "largest" else np.sort(p.lam)[: p.k]
    m = O.eig_metrics(p.A, res.lam.cpu().numpy(), res.V.cpu().numpy(), true)
    assert m["lam_err"] <= 1e-12 and m["orth"] <= 5e-15 * 512 and m["resid"] <= 1e-13, m
    check_schedule(res.info, 0.2, r)
    assert res.info["zolo_steps"] == (3 if r == 1 else 2)
    assert res.info["it_qr"] == (0 if r == 1 else 1), res.info
    assert res.info["it_chol"] == (3 if r == 1 else 2 * r - res.info["it_qr"]), res.info


@pytest.mark.parametrize("r,frac,decades", [(2, 0.05, 12.0), (4, 0.25, 12.0), (8, 0.25, 12.0)])
def test_svd_zolo(Q, r, frac, decades):
    """700 x 500: top 5 % (s ~ 0.5, Cholesky terms only) and top 25 % of 12 decades
    (s ~ 1e-3: the small shifts take the QR form)."""
    q = I.svd_logspaced(700, 500, 2000 + r, frac, decades)
    res = Q.svd(dev(q.A), k=q.k, zolo_r=r)
    mt = O.svd_metrics(q.A, res.sigma.cpu().numpy(), res.U.cpu().numpy(), res.V.cpu().numpy(), q.sigma[: q.k])
    assert mt["sigma_err"] <= 1e-12, mt
    assert mt["orthU"] <= 5e-15 * 500 and mt["orthV"] <= 5e-15 * 500, mt
    assert mt["residV"] <= 1e-13 and mt["residU"] <= 1e-13, mt
    check_schedule(res.info, res.info["s"], r)
    if frac == 0.25:
        assert res.info["it_qr"] >= 1, res.info


def test_zolo_emulated_and_option_checks(Q):
    """Zolo-PD with emulated FP64 products meets the FP64 tolerances; with FP32 Cholesky
    steps (QDWHP_MIXED) it is refused before anything runs."""
    p = I.eig_uniform(1024, 77, 0.10)
    res = Q.eig(dev(p.A), k=p.k, zolo_r=2, precision=Q.FP64_EMULATED)
    m = O.eig_metrics(p.A, res.lam.cpu().numpy(), res.V.cpu().numpy(), np.sort(p.lam)[::-1][: p.k])
    assert m["lam_err"] <= 1e-12 and m["orth"] <= 5e-15 * 1024 and m["resid"] <= 1e-13, m
    with pytest.raises(Q.QdwhpError) as e:
        Q.eig(dev(p.A), k=p.k, zolo_r=2, precision=Q.MIXED)
    assert e.value.status == -1
    with pytest.raises(Q.QdwhpError) as e:
        Q.eig(dev(p.A), k=p.k, zolo_r=9)
    assert e.value.status == -1


def test_r1_schedule_matches_qdwh_at_small_threshold(Q):
    """The 20 largest singular values log-spaced from 1 to 1e-9 above 380 in [1e-11, 1e-10]:
    the threshold for k = 20 is near 1e-9, and Zolo-PD with r = 1 must follow QDWH's ell_k,
    whose weights are algebraic (Section 3.1), to 1e-13 relative.  This pins the device's
    elliptic functions where the modulus is within 1e-18 of 1."""
    rng = np.random.default_rng(61)
    sig = np.concatenate([np.logspace(0.0, -9.0, 20), np.logspace(-10.0, -11.0, 380)])
    A = I.general_with_singular_values(500, sig, rng)
    rz = Q.svd(dev(A), k=20, zolo_r=1)
    rq = Q.svd(dev(A), k=20)
    assert rz.info["s"] == rq.info["s"] and rz.info["s"] < 1e-8, (rz.info["s"], rq.info["s"])
    ez, eq = np.array(rz.info["ell_k"]), np.array(rq.info["ell_k"])
    assert ez.size == eq.size >= 5, (ez, eq)
    assert np.all(np.abs(ez - eq) <= 1e-13 * eq), (ez, eq)
    for r in (rz, rq):
        mt = O.svd_metrics(A, r.sigma.cpu().numpy(), r.U.cpu().numpy(), r.V.cpu().numpy(), sig[:20])
        assert mt["sigma_err"] <= 1e-12, mt
