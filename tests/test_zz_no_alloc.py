"""qdwhp_potrf_f64_noalloc: the Cholesky factorisation for callers that cannot give the
library device scratch (their device memory is managed by someone else's allocator,
or a cudaMalloc on their path is not allowed).  It must give the same factor as
qdwhp_potrf_f64, which takes a caller-provided workspace, call after call, although
every call reuses the same library-owned scratch array.

Kept in a file that pytest collects last, so a stop at the first failure has already
run every other test."""

import ctypes as C

import numpy as np
import pytest

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


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n))
    return G @ G.T / n + np.eye(n)


def _noalloc(Q, Z):
    n = Z.shape[0]
    Zc = torch.from_numpy(np.asfortranarray(Z).T.copy()).to("cuda")   # column-major storage
    info = C.c_int(-1)
    st = Q.lib().qdwhp_potrf_f64_noalloc(n, Zc.data_ptr(), n, C.byref(info),
                                         torch.cuda.current_stream().cuda_stream)
    return st, info.value, torch.tril(Zc.t()).cpu().numpy()


def test_noalloc_matches_workspace_version_twice(Q):
    n = 1000
    for call, seed in enumerate((11, 12)):          # two calls in a row on the shared scratch
        Z = _spd(n, seed)
        L_ref, info_ref = Q.potrf_f64(torch.from_numpy(Z).to("cuda"))
        st, info, L = _noalloc(Q, Z)
        assert st == 0 and info == 0 and info_ref == 0, call
        L_ref = L_ref.cpu().numpy()
        # same tolerance as the workspace version's own test against LAPACK
        assert np.linalg.norm(L - L_ref) <= 1e-13 * np.linalg.norm(L_ref), call
        assert np.linalg.norm(L @ L.T - Z) <= 1e-14 * n * np.linalg.norm(Z), call


def test_noalloc_breakdown_flag_starts_clean(Q):
    n = 300
    Z = np.eye(n)
    Z[200, 200] = -1.0
    st, info, _ = _noalloc(Q, Z)
    assert st == -4 and info == 201
    # the next call must not see the previous failure
    st, info, L = _noalloc(Q, _spd(n, 3))
    assert st == 0 and info == 0


def test_noalloc_allocates_no_device_memory(Q):
    """The property the entry point exists for: after a warm-up call, further calls change
    neither the device's free memory (cudaMemGetInfo) nor torch's allocator statistics."""
    n = 2048
    Z = _spd(n, 21)
    Zc = torch.from_numpy(np.asfortranarray(Z).T.copy()).to("cuda")
    work = Zc.clone()
    info = C.c_int(-1)
    stream = torch.cuda.current_stream().cuda_stream
    assert Q.lib().qdwhp_potrf_f64_noalloc(n, work.data_ptr(), n, C.byref(info), stream) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for _ in range(3):
        work.copy_(Zc)
        assert Q.lib().qdwhp_potrf_f64_noalloc(n, work.data_ptr(), n, C.byref(info), stream) == 0
        assert info.value == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == alloc0


@pytest.mark.parametrize("n,bad", [(300, 128), (4096, 64 * 40), (4096, 4095)])
def test_noalloc_breakdown_on_split_boundaries_and_at_the_limit(Q, n, bad):
    """A failing pivot on a recursion split (a multiple of the 64-wide leaf), and at the largest
    order the static scratch takes; a successful call right after a failing one gives the same
    factor as qdwhp_potrf_f64."""
    Z = _spd(n, 5)
    Z[bad, :] = 0.0
    Z[:, bad] = 0.0
    Z[bad, bad] = -1.0
    st, info, _ = _noalloc(Q, Z)
    assert st == -4 and info == bad + 1
    Z2 = _spd(n, 6)
    st, info, L = _noalloc(Q, Z2)
    assert st == 0 and info == 0
    L_ref, info_ref = Q.potrf_f64(torch.from_numpy(Z2).to("cuda"))
    assert info_ref == 0
    L_ref = L_ref.cpu().numpy()
    assert np.linalg.norm(L - L_ref) <= 1e-13 * np.linalg.norm(L_ref)


def test_noalloc_rejects_oversize(Q):
    n = 4097
    fake = C.c_void_p(0x1000)
    info = C.c_int(-1)
    st = Q.lib().qdwhp_potrf_f64_noalloc(n, fake, n, C.byref(info), None)
    assert st == -1
    assert b"4096" in Q.lib().qdwhp_last_error_message()
