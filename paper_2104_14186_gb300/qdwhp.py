"""Python binding of the qdwhp C ABI (include/qdwhp.h).

Argument marshalling only: every step of a solve runs in libqdwhp.so's CUDA
kernels.  PyTorch supplies device memory (inputs, outputs and the workspace the
library asks for) and the current CUDA stream.  Matrices cross the boundary in
column-major order: a logical torch matrix ``A`` is passed as the storage of
``A.t().contiguous()``, and outputs are allocated transposed and returned as
``.t()`` views.

If the compiled library is missing the import of this module fails: there is no
CPU fallback.
"""

from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libqdwhp.so")

QDWHP_OK = 0
QDWHP_PENDING = 1
STATUS_NAMES = {
    0: "OK", -1: "ERR_ARG", -2: "ERR_NOMEM", -3: "ERR_NOT_CONVERGED", -4: "ERR_BREAKDOWN",
    -5: "ERR_NONFINITE", -6: "ERR_TIMEOUT", -7: "ERR_CUDA", -8: "ERR_QUEUE_FULL", -9: "ERR_COUNT", 1: "PENDING",
}
LARGEST, SMALLEST = 0, 1
FP64, MIXED, FP64_EMULATED, MIXED_EMULATED = 0, 1, 2, 3


class Opts(C.Structure):
    _fields_ = [
        ("count", C.c_int64), ("fraction", C.c_double), ("side", C.c_int32), ("precision", C.c_int32),
        ("s_eig", C.c_double), ("iters_eig", C.c_int32), ("lanczos_steps", C.c_int32), ("tol", C.c_double),
        ("c_qr", C.c_double), ("block_extra", C.c_int32), ("power_steps", C.c_int32), ("guard", C.c_double),
        ("max_retries", C.c_int32), ("jacobi_max_sweeps", C.c_int32), ("seed", C.c_uint64),
        ("refine_steps", C.c_int32), ("zolo_r", C.c_int32), ("use_omega", C.c_int32), ("zolo_c_qr", C.c_double),
    ]


class Info(C.Structure):
    _fields_ = [
        ("it_qr", C.c_int32), ("it_chol", C.c_int32), ("retries", C.c_int32), ("jacobi_sweeps", C.c_int32),
        ("ell", C.c_int64), ("k", C.c_int64), ("t", C.c_double), ("mu", C.c_double), ("s", C.c_double),
        ("alpha", C.c_double), ("ell_k", C.c_double * 12), ("conv", C.c_double * 12), ("ms_total", C.c_float),
        ("it_f32", C.c_int32), ("dc_nodes", C.c_int32), ("zolo_steps", C.c_int32),
    ]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("ell_k", "conv")}
        n = self.zolo_steps if self.zolo_steps else self.it_qr + self.it_chol
        d["ell_k"] = list(self.ell_k)[:n]
        d["conv"] = list(self.conv)[:n]
        return d


class SyevInfo(C.Structure):
    _fields_ = [
        ("nodes", C.c_int32), ("leaves", C.c_int32), ("depth", C.c_int32), ("qdwh_steps", C.c_int32),
        ("refinements", C.c_int32), ("jacobi_sweeps", C.c_int32), ("max_offblock", C.c_double),
        ("ms_total", C.c_float), ("median_splits", C.c_int32),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class GesvdInfo(C.Structure):
    _fields_ = [
        ("it_qr", C.c_int32), ("it_chol", C.c_int32), ("nodes", C.c_int32), ("leaves", C.c_int32),
        ("depth", C.c_int32), ("jacobi_sweeps", C.c_int32), ("orthonormalized", C.c_int32),
        ("median_splits", C.c_int32), ("alpha", C.c_double), ("max_offblock", C.c_double), ("ms_total", C.c_float),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class QdwhpError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = f"{where}: {STATUS_NAMES.get(status, status)}"
        if status == -7:
            msg += " (" + lib().qdwhp_last_error_message().decode() + ")"
        super().__init__(msg)
        self.status = status


_lib = None

P = C.c_void_p
I64 = C.c_int64
D = C.c_double
SIGNATURES = {
    "qdwhp_default_opts": (None, [C.POINTER(Opts)]),
    "qdwhp_status_string": (C.c_char_p, [C.c_int]),
    "qdwhp_last_error_message": (C.c_char_p, []),
    "qdwhp_k_from_fraction": (I64, [I64, D]),
    "qdwhp_eig_workspace_bytes": (C.c_size_t, [I64, C.POINTER(Opts)]),
    "qdwhp_eig": (C.c_int, [P, I64, I64, C.POINTER(Opts), P, P, I64, P, C.c_size_t, C.POINTER(Info), P]),
    "qdwhp_svd_workspace_bytes": (C.c_size_t, [I64, I64, C.POINTER(Opts)]),
    "qdwhp_svd": (C.c_int, [P, I64, I64, I64, I64, C.POINTER(Opts), P, P, I64, P, I64, P, C.c_size_t,
                            C.POINTER(Info), P]),
    "qdwhp_eig_host_workspace_bytes": (C.c_size_t, [I64, C.POINTER(Opts)]),
    "qdwhp_eig_host": (C.c_int, [P, I64, I64, C.POINTER(Opts), P, P, I64, P, C.c_size_t, C.POINTER(Info), P]),
    "qdwhp_svd_host_workspace_bytes": (C.c_size_t, [I64, I64, I64, C.POINTER(Opts)]),
    "qdwhp_svd_host": (C.c_int, [P, I64, I64, I64, I64, C.POINTER(Opts), P, P, I64, P, I64, P, C.c_size_t,
                                 C.POINTER(Info), P]),
    "qdwhp_syev_workspace_bytes": (C.c_size_t, [I64]),
    "qdwhp_syev_f64": (C.c_int, [P, I64, I64, P, P, I64, P, C.c_size_t, C.POINTER(SyevInfo), P]),
    "qdwhp_gesvd_workspace_bytes": (C.c_size_t, [I64, I64, C.c_int32]),
    "qdwhp_gesvd_f64": (C.c_int, [P, I64, I64, I64, C.c_int32, P, P, I64, P, I64, P, C.c_size_t,
                                  C.POINTER(GesvdInfo), P]),
    "qdwhp_gemm_f64_emulated_workspace_bytes": (C.c_size_t, [I64, I64, I64]),
    "qdwhp_gemm_f64_emulated": (C.c_int, [C.c_int, C.c_int, I64, I64, I64, D, P, I64, P, I64, D, P, I64, P,
                                          C.c_size_t, P]),
    "qdwhp_gemm_f64": (C.c_int, [C.c_int, C.c_int, I64, I64, I64, D, P, I64, P, I64, D, P, I64, P]),
    "qdwhp_gemm_f32_bf16x6_workspace_bytes": (C.c_size_t, [I64, I64, I64]),
    "qdwhp_gemm_f32_bf16x6": (C.c_int, [C.c_int, C.c_int, I64, I64, I64, C.c_float, P, I64, P, I64, C.c_float, P,
                                        I64, P, C.c_size_t, P]),
    "qdwhp_potrf_workspace_bytes": (C.c_size_t, [I64]),
    "qdwhp_potrf_f64": (C.c_int, [I64, P, I64, P, C.c_size_t, C.POINTER(C.c_int), P]),
    "qdwhp_qr_workspace_bytes": (C.c_size_t, [I64, I64]),
    "qdwhp_qr_f64": (C.c_int, [I64, I64, P, I64, P, I64, P, I64, P, C.c_size_t, P]),
    "qdwhp_qdwh_workspace_bytes": (C.c_size_t, [I64, I64]),
    "qdwhp_qdwh_steps_f64": (C.c_int, [I64, I64, P, I64, C.c_int32, C.POINTER(D), C.POINTER(C.c_int32),
                                       C.POINTER(D), P, C.c_size_t, P]),
    "qdwhp_potrf_f64_noalloc": (C.c_int, [I64, P, I64, C.POINTER(C.c_int), P]),
    "qdwhp_queue_create": (C.c_int, [C.c_size_t, C.c_int32, P, C.POINTER(P)]),
    "qdwhp_submit_eig": (C.c_int, [P, P, I64, I64, C.POINTER(Opts), P, P, I64, P, C.POINTER(C.c_uint64)]),
    "qdwhp_submit_svd": (C.c_int, [P, P, I64, I64, I64, I64, C.POINTER(Opts), P, P, I64, P, I64, P,
                                   C.POINTER(C.c_uint64)]),
    "qdwhp_poll": (C.c_int, [P, C.c_uint64, C.POINTER(Info)]),
    "qdwhp_wait": (C.c_int, [P, C.c_uint64, C.c_int32, C.POINTER(Info)]),
    "qdwhp_request_times": (C.c_int, [P, C.c_uint64, C.POINTER(D), C.POINTER(D), C.POINTER(D)]),
    "qdwhp_release": (C.c_int, [P, C.c_uint64]),
    "qdwhp_queue_destroy": (C.c_int, [P]),
    "qdwhp_eig_batched": (C.c_int, [I64, C.POINTER(P), C.POINTER(I64), C.POINTER(I64), C.POINTER(Opts),
                                    C.POINTER(P), C.POINTER(P), C.POINTER(I64), C.c_int32, C.POINTER(C.c_int),
                                    C.POINTER(Info), P]),
    "qdwhp_tune_set": (C.c_int, [C.c_int32, C.c_int32, C.c_int32]),
    "qdwhp_tune_get": (C.c_int32, [C.c_int32, C.c_int32]),
    "qdwhp_tune_reset": (None, []),
    "qdwhp_launch_count": (C.c_ulonglong, []),
    "qdwhp_profile_begin": (C.c_int, []),
    "qdwhp_profile_end": (C.c_int, [C.POINTER(D), C.POINTER(D), C.POINTER(I64)]),
    "qdwhp_profile_records": (I64, [C.POINTER(D), I64]),
}


def lib():
    """The loaded libqdwhp.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2104_14186_gb300.build.build() "
                               "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int, where: str):
    if status != QDWHP_OK:
        raise QdwhpError(status, where)


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _colmajor(A: torch.Tensor) -> torch.Tensor:
    """Storage holding the logical matrix A in column-major order (ld = rows)."""
    if A.dtype != torch.float64 or not A.is_cuda or A.dim() != 2:
        raise ValueError("expected a 2-D float64 CUDA tensor")
    return A.t().contiguous()


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().qdwhp_default_opts(C.byref(o))
    side = kw.pop("side", None)
    if side is not None:
        o.side = SMALLEST if str(side).lower().startswith("s") else LARGEST
    for key, val in kw.items():
        if not hasattr(o, key):
            raise TypeError(f"unknown option {key}")
        setattr(o, key, val)
    return o


def k_from_fraction(n: int, fraction: float) -> int:
    return int(lib().qdwhp_k_from_fraction(n, fraction))


def workspace(nbytes: int, device=None) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device or "cuda")


@dataclass
class EigResult:
    lam: torch.Tensor      # (k,)
    V: torch.Tensor        # (n, k)
    info: dict


@dataclass
class SvdResult:
    sigma: torch.Tensor    # (k,)
    U: torch.Tensor        # (m, k)
    V: torch.Tensor        # (n, k)
    info: dict


def _host_colmajor(A: torch.Tensor) -> torch.Tensor:
    """Column-major storage of a host float64 matrix: A's own storage when it is already
    column-major (A.t() contiguous), else a copy."""
    if A.dtype != torch.float64 or A.is_cuda or A.dim() != 2:
        raise ValueError("expected a 2-D float64 host tensor")
    At = A.t()
    return At if At.is_contiguous() else At.contiguous()


def _host_out(shape, pin: bool) -> torch.Tensor:
    return torch.empty(shape, dtype=torch.float64, pin_memory=pin)


def eig(A: torch.Tensor, k: int | None = None, fraction: float | None = None, side: str = "largest",
        ws: torch.Tensor | None = None, stream=None, device=None, out=None, **opts) -> EigResult:
    """qdwhp_eig: k largest (or smallest) eigenpairs of the symmetric float64 matrix A.

    A CUDA tensor is solved on its device.  A host tensor goes through qdwhp_eig_host (the
    library copies A in and lambda, V out on the stream of `device`, default cuda:0); `out`
    may hold preallocated host tensors (lambda (k,), V^T (k, n)), pinned for asynchronous
    copies."""
    n = A.shape[0]
    if A.shape != (n, n):
        raise ValueError("A must be square")
    o = default_opts(side=side, **opts)
    if k is not None:
        o.count = int(k)
    elif fraction is not None:
        o.count = 0
        o.fraction = float(fraction)
    kk = int(o.count) if o.count > 0 else k_from_fraction(n, o.fraction)
    if not A.is_cuda:
        dev = torch.device(device or "cuda")
        Ac = _host_colmajor(A)
        lam, Vt = out if out is not None else (_host_out(max(kk, 1), Ac.is_pinned()),
                                               _host_out((max(kk, 1), n), Ac.is_pinned()))
        need = lib().qdwhp_eig_host_workspace_bytes(n, C.byref(o))
        if need == 0:
            raise QdwhpError(-1, "qdwhp_eig_host_workspace_bytes")
        if ws is None or ws.numel() < need:
            ws = workspace(need, dev)
        info = Info()
        st = stream if stream is not None else torch.cuda.current_stream(dev)
        rc = lib().qdwhp_eig_host(_ptr(Ac), n, n, C.byref(o), _ptr(lam), _ptr(Vt), n, _ptr(ws), ws.numel(),
                                  C.byref(info), st.cuda_stream)
        _check(rc, "qdwhp_eig_host")
        return EigResult(lam[:kk], Vt[:kk].t(), info.as_dict())
    Ac = _colmajor(A)
    lam = torch.empty(max(kk, 1), dtype=torch.float64, device=A.device)
    Vt = torch.empty(max(kk, 1), n, dtype=torch.float64, device=A.device)
    need = lib().qdwhp_eig_workspace_bytes(n, C.byref(o))
    if ws is None or ws.numel() < need:
        ws = workspace(need, A.device)
    info = Info()
    st = lib().qdwhp_eig(_ptr(Ac), n, n, C.byref(o), _ptr(lam), _ptr(Vt), n, _ptr(ws), ws.numel(), C.byref(info),
                         _stream(stream))
    _check(st, "qdwhp_eig")
    return EigResult(lam[:kk], Vt[:kk].t(), info.as_dict())


def syev(A: torch.Tensor, ws: torch.Tensor | None = None, stream=None):
    """qdwhp_syev_f64: all eigenpairs of the symmetric CUDA float64 matrix A (ascending).
    Returns (lam, V, info dict)."""
    n = A.shape[0]
    if A.shape != (n, n):
        raise ValueError("A must be square")
    Ac = _colmajor(A)
    lam = torch.empty(n, dtype=torch.float64, device=A.device)
    Vt = torch.empty(n, n, dtype=torch.float64, device=A.device)
    need = lib().qdwhp_syev_workspace_bytes(n)
    if ws is None or ws.numel() < need:
        ws = workspace(need, A.device)
    info = SyevInfo()
    st = lib().qdwhp_syev_f64(_ptr(Ac), n, n, _ptr(lam), _ptr(Vt), n, _ptr(ws), ws.numel(), C.byref(info),
                              _stream(stream))
    _check(st, "qdwhp_syev_f64")
    return lam, Vt.t(), info.as_dict()


def gesvd(A: torch.Tensor, precision: int = 0, ws: torch.Tensor | None = None, stream=None):
    """qdwhp_gesvd_f64: all singular triplets (thin, p = min(m, n)) of the CUDA float64
    matrix A by QDWH-SVD.  precision: FP64 or FP64_EMULATED.  Returns (sigma descending,
    U m x p, V n x p, info dict)."""
    m, n = A.shape
    p = min(m, n)
    Ac = _colmajor(A)
    sig = torch.empty(p, dtype=torch.float64, device=A.device)
    Ut = torch.empty(p, m, dtype=torch.float64, device=A.device)
    Vt = torch.empty(p, n, dtype=torch.float64, device=A.device)
    need = lib().qdwhp_gesvd_workspace_bytes(m, n, precision)
    if need == 0:
        raise QdwhpError(-1, "qdwhp_gesvd_workspace_bytes")
    if ws is None or ws.numel() < need:
        ws = workspace(need, A.device)
    info = GesvdInfo()
    st = lib().qdwhp_gesvd_f64(_ptr(Ac), m, n, m, precision, _ptr(sig), _ptr(Ut), m, _ptr(Vt), n, _ptr(ws),
                               ws.numel(), C.byref(info), _stream(stream))
    _check(st, "qdwhp_gesvd_f64")
    return sig, Ut.t(), Vt.t(), info.as_dict()


def svd(A: torch.Tensor, k: int | None = None, fraction: float | None = None, ws: torch.Tensor | None = None,
        stream=None, device=None, out=None, **opts) -> SvdResult:
    """qdwhp_svd: k largest singular triplets of the float64 matrix A (m x n).

    A CUDA tensor is solved in place on its device.  A host tensor goes through
    qdwhp_svd_host: the library copies A to `device` (default cuda:0), solves, and copies
    sigma, U and V back into host tensors on the stream before returning; `out` may hold
    preallocated host tensors (sigma (k,), U^T (k, m), V^T (k, n)), pinned for asynchronous
    copies.
    """
    m, n = A.shape
    o = default_opts(**opts)
    kk = 0
    if k is not None:
        kk = int(k)
    elif fraction is not None:
        o.fraction = float(fraction)
    kres = kk if kk > 0 else (int(o.count) if o.count > 0 else k_from_fraction(min(m, n), o.fraction))
    if not A.is_cuda:
        dev = torch.device(device or "cuda")
        Ac = _host_colmajor(A)
        pin = Ac.is_pinned()
        sig, Ut, Vt = out if out is not None else (_host_out(max(kres, 1), pin), _host_out((max(kres, 1), m), pin),
                                                   _host_out((max(kres, 1), n), pin))
        need = lib().qdwhp_svd_host_workspace_bytes(m, n, kk, C.byref(o))
        if need == 0:
            raise QdwhpError(-1, "qdwhp_svd_host_workspace_bytes")
        if ws is None or ws.numel() < need:
            ws = workspace(need, dev)
        info = Info()
        st = stream if stream is not None else torch.cuda.current_stream(dev)
        rc = lib().qdwhp_svd_host(_ptr(Ac), m, n, m, kk, C.byref(o), _ptr(sig), _ptr(Ut), m, _ptr(Vt), n, _ptr(ws),
                                  ws.numel(), C.byref(info), st.cuda_stream)
        _check(rc, "qdwhp_svd_host")
        return SvdResult(sig[:kres], Ut[:kres].t(), Vt[:kres].t(), info.as_dict())
    with torch.cuda.stream(stream) if stream is not None else _nullctx():
        Ac = _colmajor(A)
        sigma = torch.empty(max(kres, 1), dtype=torch.float64, device=A.device)
        Ut = torch.empty(max(kres, 1), m, dtype=torch.float64, device=A.device)
        Vt = torch.empty(max(kres, 1), n, dtype=torch.float64, device=A.device)
        need = lib().qdwhp_svd_workspace_bytes(m, n, C.byref(o))
        if ws is None or ws.numel() < need:
            ws = workspace(need, A.device)
        info = Info()
        st = lib().qdwhp_svd(_ptr(Ac), m, n, m, kk, C.byref(o), _ptr(sigma), _ptr(Ut), m, _ptr(Vt), n, _ptr(ws),
                             ws.numel(), C.byref(info), _stream(stream))
    _check(st, "qdwhp_svd")
    return SvdResult(sigma[:kres], Ut[:kres].t(), Vt[:kres].t(), info.as_dict())


class _nullctx:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


class Queue:
    """qdwhp_queue: serving queue with HBM-budget admission (argument marshalling only).

    Keeps the tensors of every request alive until it is released."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 4):
        self.h = P()
        _check(lib().qdwhp_queue_create(int(hbm_budget_bytes), int(max_slots), None, C.byref(self.h)),
               "qdwhp_queue_create")
        self.keep = {}

    def submit_eig(self, A: torch.Tensor, k: int, side: str = "largest", stream=None, **opts) -> int:
        n = A.shape[0]
        o = default_opts(side=side, **opts)
        o.count = int(k)
        Ac = _colmajor(A)
        lam = torch.empty(k, dtype=torch.float64, device=A.device)
        Vt = torch.empty(k, n, dtype=torch.float64, device=A.device)
        rid = C.c_uint64(0)
        _check(lib().qdwhp_submit_eig(self.h, _ptr(Ac), n, n, C.byref(o), _ptr(lam), _ptr(Vt), n, _stream(stream),
                                      C.byref(rid)), "qdwhp_submit_eig")
        self.keep[rid.value] = ("eig", Ac, lam, Vt, o)
        return rid.value

    def submit_svd(self, A: torch.Tensor, k: int, stream=None, **opts) -> int:
        m, n = A.shape
        o = default_opts(**opts)
        Ac = _colmajor(A)
        sig = torch.empty(k, dtype=torch.float64, device=A.device)
        Ut = torch.empty(k, m, dtype=torch.float64, device=A.device)
        Vt = torch.empty(k, n, dtype=torch.float64, device=A.device)
        rid = C.c_uint64(0)
        _check(lib().qdwhp_submit_svd(self.h, _ptr(Ac), m, n, m, int(k), C.byref(o), _ptr(sig), _ptr(Ut), m, _ptr(Vt),
                                      n, _stream(stream), C.byref(rid)), "qdwhp_submit_svd")
        self.keep[rid.value] = ("svd", Ac, sig, Ut, Vt, o)
        return rid.value

    def poll(self, rid: int) -> int:
        return int(lib().qdwhp_poll(self.h, rid, None))

    def wait(self, rid: int, timeout_ms: int = 600000):
        info = Info()
        st = lib().qdwhp_wait(self.h, rid, int(timeout_ms), C.byref(info))
        _check(st, "qdwhp_wait")
        kept = self.keep[rid]
        if kept[0] == "eig":
            return EigResult(kept[2], kept[3].t(), info.as_dict())
        return SvdResult(kept[2], kept[3].t(), kept[4].t(), info.as_dict())

    def times(self, rid: int):
        a, b, c = D(0), D(0), D(0)
        lib().qdwhp_request_times(self.h, rid, C.byref(a), C.byref(b), C.byref(c))
        return a.value, b.value, c.value

    def release(self, rid: int):
        lib().qdwhp_release(self.h, rid)
        self.keep.pop(rid, None)

    def close(self):
        if self.h:
            _check(lib().qdwhp_queue_destroy(self.h), "qdwhp_queue_destroy")
            self.h = P()
            self.keep.clear()


def eig_batched(As, ks_fraction: float = 0.1, concurrency: int = 8, side: str = "largest", **opts):
    """qdwhp_eig_batched over a list of symmetric CUDA float64 matrices; returns (results, statuses)."""
    cnt = len(As)
    o = default_opts(side=side, **opts)
    o.count = 0
    o.fraction = float(ks_fraction)
    cols = [_colmajor(A) for A in As]
    ns = [A.shape[0] for A in As]
    kk = [k_from_fraction(n, ks_fraction) for n in ns]
    lams = [torch.empty(k, dtype=torch.float64, device=A.device) for k, A in zip(kk, As)]
    Vts = [torch.empty(k, n, dtype=torch.float64, device=A.device) for k, n, A in zip(kk, ns, As)]
    Pa = (P * cnt)(*[_ptr(c) for c in cols])
    Pl = (P * cnt)(*[_ptr(x) for x in lams])
    Pv = (P * cnt)(*[_ptr(x) for x in Vts])
    Na = (I64 * cnt)(*ns)
    sts = (C.c_int * cnt)()
    infos = (Info * cnt)()
    lib().qdwhp_eig_batched(cnt, Pa, Na, Na, C.byref(o), Pl, Pv, Na, int(concurrency), sts, infos, _stream(None))
    res = [EigResult(lams[i], Vts[i].t(), infos[i].as_dict()) for i in range(cnt)]
    return res, [int(sts[i]) for i in range(cnt)]


def launch_count() -> int:
    return int(lib().qdwhp_launch_count())


def profile_begin():
    _check(lib().qdwhp_profile_begin(), "qdwhp_profile_begin")


def profile_end() -> dict:
    ms, fl, n = D(0.0), D(0.0), I64(0)
    _check(lib().qdwhp_profile_end(C.byref(ms), C.byref(fl), C.byref(n)), "qdwhp_profile_end")
    return {"gemm_ms": ms.value, "gemm_flops": fl.value, "gemm_launches": n.value}


def profile_records() -> list:
    n = int(lib().qdwhp_profile_records(None, 0))
    buf = (D * (6 * max(n, 1)))()
    lib().qdwhp_profile_records(buf, n)
    return [tuple(buf[6 * i:6 * i + 6]) for i in range(n)]


# ---- building blocks ----

def gemm_f64(A: torch.Tensor, B: torch.Tensor, transa=False, transb=False, alpha=1.0, beta=0.0,
             Cmat: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """C = alpha op(A) op(B) + beta C through qdwhp_gemm_f64 (logical row-major tensors in/out)."""
    Ac, Bc = _colmajor(A), _colmajor(B)
    m = A.shape[1] if transa else A.shape[0]
    k = A.shape[0] if transa else A.shape[1]
    n = B.shape[0] if transb else B.shape[1]
    Ct = (torch.zeros(n, m, dtype=torch.float64, device=A.device) if Cmat is None else _colmajor(Cmat))
    st = lib().qdwhp_gemm_f64(int(transa), int(transb), m, n, k, alpha, _ptr(Ac), A.shape[0], _ptr(Bc), B.shape[0],
                              beta, _ptr(Ct), m, _stream(stream))
    _check(st, "qdwhp_gemm_f64")
    return Ct.t()


def gemm_f64_emulated(A: torch.Tensor, B: torch.Tensor, transa=False, transb=False, alpha=1.0, beta=0.0,
                      Cmat: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """The same product through qdwhp_gemm_f64_emulated (Ozaki split on the BF16 tensor cores)."""
    Ac, Bc = _colmajor(A), _colmajor(B)
    m = A.shape[1] if transa else A.shape[0]
    k = A.shape[0] if transa else A.shape[1]
    n = B.shape[0] if transb else B.shape[1]
    Ct = (torch.zeros(n, m, dtype=torch.float64, device=A.device) if Cmat is None else _colmajor(Cmat))
    need = lib().qdwhp_gemm_f64_emulated_workspace_bytes(m, n, k)
    ws = workspace(max(need, 1), A.device)
    st = lib().qdwhp_gemm_f64_emulated(int(transa), int(transb), m, n, k, alpha, _ptr(Ac), A.shape[0], _ptr(Bc),
                                       B.shape[0], beta, _ptr(Ct), m, _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "qdwhp_gemm_f64_emulated")
    return Ct.t()


def gemm_f32_bf16x6(A: torch.Tensor, B: torch.Tensor, transa=False, transb=False, alpha=1.0, beta=0.0,
                    Cmat: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """C = alpha op(A) op(B) + beta C in FP32 through qdwhp_gemm_f32_bf16x6 (three BF16 slices per
    operand on the tensor cores); logical row-major float32 CUDA tensors in and out."""
    if A.dtype != torch.float32 or B.dtype != torch.float32 or not A.is_cuda or not B.is_cuda:
        raise ValueError("expected float32 CUDA tensors")
    Ac, Bc = A.t().contiguous(), B.t().contiguous()
    m = A.shape[1] if transa else A.shape[0]
    k = A.shape[0] if transa else A.shape[1]
    n = B.shape[0] if transb else B.shape[1]
    Ct = (torch.zeros(n, m, dtype=torch.float32, device=A.device) if Cmat is None else Cmat.t().contiguous())
    need = lib().qdwhp_gemm_f32_bf16x6_workspace_bytes(m, n, k)
    ws = workspace(max(need, 1), A.device)
    st = lib().qdwhp_gemm_f32_bf16x6(int(transa), int(transb), m, n, k, alpha, _ptr(Ac), A.shape[0], _ptr(Bc),
                                     B.shape[0], beta, _ptr(Ct), m, _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "qdwhp_gemm_f32_bf16x6")
    return Ct.t()


def potrf_f64(Z: torch.Tensor, stream=None):
    """Lower Cholesky factor L (Z = L L^T) through qdwhp_potrf_f64; returns (L, info)."""
    n = Z.shape[0]
    Zc = _colmajor(Z)
    ws = workspace(lib().qdwhp_potrf_workspace_bytes(n), Z.device)
    info = C.c_int(0)
    st = lib().qdwhp_potrf_f64(n, _ptr(Zc), n, _ptr(ws), ws.numel(), C.byref(info), _stream(stream))
    if st not in (QDWHP_OK, -4):
        _check(st, "qdwhp_potrf_f64")
    return torch.tril(Zc.t()), info.value


def qr_f64(A: torch.Tensor, stream=None):
    """Householder QR A = Q R (m >= n) through qdwhp_qr_f64; returns (Q, R)."""
    m, n = A.shape
    Ac = _colmajor(A)
    Qt = torch.empty(n, m, dtype=torch.float64, device=A.device)
    Rt = torch.empty(n, n, dtype=torch.float64, device=A.device)
    ws = workspace(lib().qdwhp_qr_workspace_bytes(m, n), A.device)
    st = lib().qdwhp_qr_f64(m, n, _ptr(Ac), m, _ptr(Qt), m, _ptr(Rt), n, _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "qdwhp_qr_f64")
    return Qt.t(), Rt.t()


def qdwh_steps_f64(X: torch.Tensor, weights, use_qr, stream=None):
    """Apply QDWH steps with the given (a, b, c) weights in place; returns (X_new, conv)."""
    m, n = X.shape
    Xc = _colmajor(X)
    ns = len(weights)
    abc = (C.c_double * (3 * max(ns, 1)))(*[float(v) for w in weights for v in w[:3]])
    uq = (C.c_int32 * max(ns, 1))(*[int(u) for u in use_qr])
    conv = (C.c_double * max(ns, 1))()
    ws = workspace(lib().qdwhp_qdwh_workspace_bytes(m, n), X.device)
    st = lib().qdwhp_qdwh_steps_f64(m, n, _ptr(Xc), m, ns, abc, uq, conv, _ptr(ws), ws.numel(), _stream(stream))
    _check(st, "qdwhp_qdwh_steps_f64")
    return Xc.t(), [conv[i] for i in range(ns)]
