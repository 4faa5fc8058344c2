"""Launch-shape knobs (qdwhp_tune_set) on the GPU: solves under extreme settings still meet
the FP64 tolerances (the knobs change launch shapes, not the computation), and the autotuner
produces a valid table."""

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
    yield qdwhp
    qdwhp.lib().qdwhp_tune_reset()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


@pytest.mark.parametrize("panel,warps,splitk", [(16, 1, 1), (512, 8, 8), (32, 16, 4)])
def test_solves_under_extreme_knobs(Q, panel, warps, splitk):
    lib = Q.lib()
    try:
        for c in range(5):
            assert lib.qdwhp_tune_set(0, c, panel) == 0
            assert lib.qdwhp_tune_set(1, c, warps) == 0
            assert lib.qdwhp_tune_set(2, c, splitk) == 0
        p = I.eig_uniform(512, 1000, 0.10)
        r = Q.eig(dev(p.A), k=p.k)
        m = O.eig_metrics(p.A, r.lam.cpu().numpy(), r.V.cpu().numpy(), np.sort(p.lam)[::-1][: p.k])
        assert m["lam_err"] <= 1e-12 and m["orth"] <= 5e-15 * 512 and m["resid"] <= 1e-13, m
        q = I.svd_logspaced(700, 500, 2000, 0.05)
        rs = Q.svd(dev(q.A), k=q.k)
        mt = O.svd_metrics(q.A, rs.sigma.cpu().numpy(), rs.U.cpu().numpy(), rs.V.cpu().numpy(), q.sigma[: q.k])
        assert mt["sigma_err"] <= 1e-12 and mt["residV"] <= 1e-13 and mt["residU"] <= 1e-13, mt
    finally:
        lib.qdwhp_tune_reset()


def test_autotuner_produces_valid_table(Q, tmp_path):
    from paper_2104_14186_gb300 import autotune
    try:
        res = autotune.tune(classes=(0, 1), reps=2)
        for name, (knob, cands) in autotune.KNOBS.items():
            vals = res["table"][name]
            assert len(vals) == 5 and vals[0] in cands and vals[1] in cands, (name, vals)
        path = str(tmp_path / "t.json")
        autotune.save(res, path)
        autotune.apply(autotune.load(path))
    finally:
        Q.lib().qdwhp_tune_reset()
