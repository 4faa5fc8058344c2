"""Serving queue and batched solves: each result is the same alone and in the mix.

Requests of mixed kinds and sizes are submitted together to a queue whose HBM budget
admits only some of them at a time, so later requests start while earlier ones run
(continuous batching); every result must equal the same problem solved alone through
qdwhp_eig / qdwhp_svd (the kernels are deterministic, so the comparison is exact), and
meet the plain-FP64 tolerances against the constructed spectra."""

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


def test_queue_results_equal_alone_and_in_the_mix(Q):
    probs = []
    for i, n in enumerate((300, 520, 180, 700, 256, 410)):
        probs.append(("eig", I.eig_uniform(n, 100 + i, 0.1, "largest" if i % 2 == 0 else "smallest")))
    for i, (m, n) in enumerate(((400, 300), (700, 350), (260, 260))):
        probs.append(("svd", I.svd_logspaced(m, n, 200 + i, 0.05 + 0.05 * i, decades=10.0)))
    budget = 3 * Q.lib().qdwhp_svd_workspace_bytes(700, 350, None)     # a few requests at a time
    q = Q.Queue(budget, max_slots=3)
    ids = []
    for kind, p in probs:
        A = dev(p.A)
        if kind == "eig":
            ids.append(q.submit_eig(A, p.k, side=p.side))
        else:
            ids.append(q.submit_svd(A, p.k))
    results = [q.wait(rid) for rid in ids]
    starts = [q.times(rid)[1] for rid in ids]
    dones = [q.times(rid)[2] for rid in ids]
    q.close()
    # continuous batching: some request started before another finished
    assert any(starts[j] < dones[i] for i in range(len(ids)) for j in range(len(ids)) if i != j)
    for (kind, p), r in zip(probs, results):
        if kind == "eig":
            alone = Q.eig(dev(p.A), k=p.k, side=p.side)
            assert torch.equal(r.lam, alone.lam) and torch.equal(r.V, alone.V)
            true = np.sort(p.lam)[::-1][: p.k] if p.side == "largest" else np.sort(p.lam)[: p.k]
            m = O.eig_metrics(p.A, r.lam.cpu().numpy(), r.V.cpu().numpy(), true)
            assert m["lam_err"] <= 1e-12 and m["resid"] <= 1e-13
        else:
            alone = Q.svd(dev(p.A), k=p.k)
            assert torch.equal(r.sigma, alone.sigma) and torch.equal(r.U, alone.U) and torch.equal(r.V, alone.V)
            m = O.svd_metrics(p.A, r.sigma.cpu().numpy(), r.U.cpu().numpy(), r.V.cpu().numpy(), p.sigma[: p.k])
            assert m["sigma_err"] <= 1e-12 and m["residU"] <= 1e-13 and m["residV"] <= 1e-13


def test_queue_admission_and_timeout(Q):
    small = Q.lib().qdwhp_eig_workspace_bytes(200, None)
    q = Q.Queue(small + (1 << 20), max_slots=1)
    p = I.eig_uniform(600, 7, 0.1)
    with pytest.raises(Q.QdwhpError) as e:          # can never fit the budget
        q.submit_eig(dev(p.A), p.k)
    assert e.value.status == -8
    p2 = I.eig_uniform(200, 8, 0.1)
    A2 = dev(p2.A)
    # The request's input is produced on this stream behind a kernel that runs for about a
    # second, so the solve cannot have finished when the zero-millisecond wait looks at it.
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        torch.cuda._sleep(2_000_000_000)
        rid = q.submit_eig(A2, p2.k, stream=side)
    info = Q.Info()
    st = Q.lib().qdwhp_wait(q.h, rid, 0, __import__("ctypes").byref(info))
    assert st == -6                                 # the bounded wait expired
    assert q.poll(rid) == 1                         # still pending
    r = q.wait(rid)
    assert r.lam.shape[0] == p2.k
    m = O.eig_metrics(p2.A, r.lam.cpu().numpy(), r.V.cpu().numpy(), np.sort(p2.lam)[::-1][: p2.k])
    assert m["lam_err"] <= 1e-12 and m["resid"] <= 1e-13
    q.close()


def test_eig_batched_matches_single_solves(Q):
    sizes = I.batch_sizes(12, 4000, 64, 400)
    probs = [I.eig_uniform(int(n), 4000 + i, 0.10) for i, n in enumerate(sizes)]
    res, sts = Q.eig_batched([dev(p.A) for p in probs], 0.10, concurrency=4)
    assert all(s == 0 for s in sts), sts
    for p, r in zip(probs, res):
        alone = Q.eig(dev(p.A), k=p.k)
        assert torch.equal(r.lam, alone.lam) and torch.equal(r.V, alone.V)
