"""The FP32-accurate BF16x6 product on the tensor cores (qdwhp_gemm_f32_bf16x6), through the C
ABI: each FP32 entry split into three bfloat16 slices, the six slice products with s + t <= 2
accumulated in FP32.  Checked against the FP64 product of the same FP32 inputs, element by
element within the FP32 rounding bound (K + 8) 2^-24 (|op(A)| |op(B)|)_ij; its root-mean-square
error within 8 times that of an FP32 product on the CUDA cores (the tensor core's FP32
accumulation is the larger part of it: before the kernel promoted its partial sums to FP32
registers every 128 of K, a 4100-deep product had 25 times the FP32 error), and at least 300
times below a plain BF16 product."""

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


def _op(X, t):
    return X.T if t else X


@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("m,n,k", [(128, 128, 128), (333, 200, 129), (1024, 768, 4100), (129, 640, 64), (5, 7, 3)])
def test_bf16x6_against_fp64_of_the_fp32_inputs(Q, ta, tb, m, n, k):
    g = torch.Generator(device="cuda").manual_seed(m * 7 + n + k + 3 * ta + tb)
    A = torch.randn(*((k, m) if ta else (m, k)), device="cuda", generator=g)
    B = torch.randn(*((n, k) if tb else (k, n)), device="cuda", generator=g)
    C0 = torch.randn(m, n, device="cuda", generator=g)
    alpha, beta = 0.75, -0.5
    C = Q.gemm_f32_bf16x6(A, B, transa=ta, transb=tb, alpha=alpha, beta=beta, Cmat=C0.clone())
    exact = alpha * (_op(A.double(), ta) @ _op(B.double(), tb)) + beta * C0.double()
    bound = (k + 8) * 2.0 ** -24 * (abs(alpha) * (_op(A.double(), ta).abs() @ _op(B.double(), tb).abs())
                                    + abs(beta) * C0.double().abs()) + 1e-30
    err = (C.double() - exact).abs()
    assert torch.all(err <= bound), float((err / bound).max())
    torch.backends.cuda.matmul.allow_tf32 = False
    ref32 = alpha * (_op(A, ta) @ _op(B, tb)) + beta * C0
    ref16 = alpha * (_op(A.bfloat16().float(), ta) @ _op(B.bfloat16().float(), tb)) + beta * C0
    rms = lambda x: float(torch.sqrt(torch.mean(x ** 2)))
    e6 = rms(C.double() - exact)
    assert e6 <= 8.0 * rms(ref32.double() - exact) + 1e-12
    assert 300.0 * e6 <= rms(ref16.double() - exact)


def test_bf16x6_beta_zero_never_reads_c_and_nan_propagates(Q):
    m = n = k = 256
    g = torch.Generator(device="cuda").manual_seed(5)
    A = torch.randn(m, k, device="cuda", generator=g)
    B = torch.randn(k, n, device="cuda", generator=g)
    Cn = torch.full((m, n), float("nan"), device="cuda")
    C = Q.gemm_f32_bf16x6(A, B, beta=0.0, Cmat=Cn)
    assert torch.isfinite(C).all()
    A[17, 3] = float("nan")
    C = Q.gemm_f32_bf16x6(A, B)
    assert torch.isnan(C[17]).all() and torch.isfinite(C[:17]).all() and torch.isfinite(C[18:]).all()


def test_mixed_solve_routes_fp32_products_to_the_tensor_cores(Q):
    """A mixed-precision EIG solve issues its FP32 products of order >= 256 as BF16x6 tensor-core
    launches (profile records marked -2), and still meets its stated accuracy."""
    from paper_2104_14186_gb300 import inputs as I
    import oracle as O
    p = I.eig_uniform(1024, 77, 0.10)
    A = torch.from_numpy(np.ascontiguousarray(p.A)).cuda()
    Q.profile_begin()
    r = Q.eig(A, k=p.k, precision=Q.MIXED)
    Q.profile_end()
    recs = Q.profile_records()
    assert sum(1 for rec in recs if rec[4] == -2) >= 2
    assert r.info["it_f32"] == 2
    m = O.eig_metrics(p.A, r.lam.cpu().numpy(), r.V.cpu().numpy(), np.sort(p.lam)[::-1][: p.k])
    assert m["lam_err"] <= 1e-6 and m["resid"] <= 1e-3 and m["orth"] <= 5e-15 * 1024, m
