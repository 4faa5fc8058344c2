"""The C-ABI library builds, loads and exports every symbol include/qdwhp.h declares;
host-only entry points behave (no GPU needed)."""

import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2104_14186_gb300 import build
    build.build()
    from paper_2104_14186_gb300 import qdwhp as Q
    return Q.lib()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "qdwhp.h")).read()
    return sorted(set(re.findall(r"QDWHP_API\s+[\w\s\*]+?\b(qdwhp_\w+)\s*\(", text)))


def test_header_declares_solvers_and_blocks():
    syms = declared_symbols()
    for name in ("qdwhp_eig", "qdwhp_svd", "qdwhp_gemm_f64", "qdwhp_potrf_f64", "qdwhp_qr_f64",
                 "qdwhp_qdwh_steps_f64", "qdwhp_default_opts"):
        assert name in syms


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_signatures_cover_header(lib):
    from paper_2104_14186_gb300 import qdwhp as Q
    assert set(declared_symbols()) <= set(Q.SIGNATURES), set(declared_symbols()) - set(Q.SIGNATURES)


def test_struct_layouts_match_header(lib):
    from paper_2104_14186_gb300 import qdwhp as Q
    o = Q.default_opts()
    assert o.s_eig == 0.2 and o.iters_eig == 3 and o.tol == 0.1 and o.c_qr == 100.0
    assert o.lanczos_steps == 30 and o.block_extra == 16 and o.power_steps == 0 and o.seed == 1234
    assert o.max_retries == 2 and o.jacobi_max_sweeps == 30 and o.side == Q.LARGEST
    assert o.use_omega == 0 and o.zolo_c_qr == 20.0 and o.zolo_r == 0 and o.refine_steps == 0


def test_k_from_fraction(lib):
    from paper_2104_14186_gb300 import inputs as I
    from paper_2104_14186_gb300 import qdwhp as Q
    for n, f in [(512, 0.10), (4096, 0.05), (16384, 0.01), (16384, 0.20), (10, 0.01), (7, 1.0)]:
        assert Q.k_from_fraction(n, f) == I.k_from_fraction(n, f)
    assert Q.k_from_fraction(512, 0.10) == 52
    assert Q.k_from_fraction(4096, 0.05) == 205
    assert Q.k_from_fraction(0, 0.1) == 0


def test_workspace_sizes_grow(lib):
    from paper_2104_14186_gb300 import qdwhp as Q
    o = Q.default_opts()
    a = lib.qdwhp_eig_workspace_bytes(512, C.byref(o))
    b = lib.qdwhp_eig_workspace_bytes(1024, C.byref(o))
    assert 0 < a < b
    assert lib.qdwhp_svd_workspace_bytes(300, 200, C.byref(o)) > 0
    # wide problems are solved transposed and need room for A^T
    assert lib.qdwhp_svd_workspace_bytes(200, 300, C.byref(o)) > lib.qdwhp_svd_workspace_bytes(300, 200, C.byref(o))


def test_svd_workspace_holds_the_reduced_route_above_512(lib):
    """Above order 512 the partial SVD's reduced problem (order ell <= n) may go to QDWH-SVD,
    so the workspace must also hold that solver's scratch for a square problem of order n."""
    from paper_2104_14186_gb300 import qdwhp as Q
    o = Q.default_opts()
    for n in (513, 1024, 3000):
        svd = lib.qdwhp_svd_workspace_bytes(n, n, C.byref(o))
        assert svd > lib.qdwhp_gesvd_workspace_bytes(n, n, 0), n
    # at or below 512 the one-sided Jacobi handles every reduced problem: no such scratch
    assert lib.qdwhp_svd_workspace_bytes(512, 512, C.byref(o)) < lib.qdwhp_gesvd_workspace_bytes(512, 512, 0)


def test_argument_errors_return_before_any_launch(lib):
    from paper_2104_14186_gb300 import qdwhp as Q
    o = Q.default_opts()
    info = Q.Info()
    fake = C.c_void_p(0x1000)
    # null A, n < 1, k > n, bad options: ERR_ARG without touching the device
    assert lib.qdwhp_eig(None, 10, 10, C.byref(o), fake, fake, 10, fake, 1 << 30, C.byref(info), None) == -1
    assert lib.qdwhp_eig(fake, 0, 10, C.byref(o), fake, fake, 10, fake, 1 << 30, C.byref(info), None) == -1
    o2 = Q.default_opts(count=11)
    assert lib.qdwhp_eig(fake, 10, 10, C.byref(o2), fake, fake, 10, fake, 1 << 30, C.byref(info), None) == -1
    o3 = Q.default_opts(s_eig=1.5)
    assert lib.qdwhp_eig(fake, 10, 10, C.byref(o3), fake, fake, 10, fake, 1 << 30, C.byref(info), None) == -1
    o4 = Q.default_opts(precision=Q.MIXED + 5)
    assert lib.qdwhp_eig(fake, 10, 10, C.byref(o4), fake, fake, 10, fake, 1 << 30, C.byref(info), None) == -1
    # workspace too small: ERR_NOMEM
    assert lib.qdwhp_eig(fake, 10, 10, C.byref(o), fake, fake, 10, fake, 16, C.byref(info), None) == -2
    assert lib.qdwhp_svd(fake, 10, 8, 10, 20, C.byref(o), fake, fake, 10, fake, 8, fake, 1 << 30,
                         C.byref(info), None) == -1
    assert lib.qdwhp_gemm_f64(0, 0, 4, 4, 4, 1.0, fake, 2, fake, 4, 0.0, fake, 4, None) == -1
    assert lib.qdwhp_qr_f64(3, 4, fake, 3, fake, 3, fake, 4, fake, 1 << 20, None) == -1


def test_status_strings(lib):
    for s in (0, -1, -2, -3, -4, -5, -6, -7, -8, -9, 1):
        assert lib.qdwhp_status_string(s)


def test_queue_argument_errors(lib):
    from paper_2104_14186_gb300 import qdwhp as Q
    h = Q.P()
    assert lib.qdwhp_queue_create(1 << 30, 0, None, C.byref(h)) == -1       # no slots
    assert lib.qdwhp_queue_create(100, 2, None, C.byref(h)) == -1           # budget too small
    assert lib.qdwhp_poll(None, 1, None) == -1
    assert lib.qdwhp_queue_destroy(None) == -1


def test_gesvd_argument_checks(lib):
    """Sizes, pointers and precision are checked before anything is launched."""
    assert lib.qdwhp_gesvd_workspace_bytes(300, 200, 0) > 0
    assert lib.qdwhp_gesvd_workspace_bytes(200, 300, 2) > lib.qdwhp_gesvd_workspace_bytes(200, 300, 0)
    assert lib.qdwhp_gesvd_workspace_bytes(300, 200, 1) == 0      # mixed is not offered
    assert lib.qdwhp_gesvd_workspace_bytes(0, 200, 0) == 0
    from paper_2104_14186_gb300 import qdwhp as Q
    info = Q.GesvdInfo()
    assert lib.qdwhp_gesvd_f64(None, 3, 3, 3, 0, None, None, 3, None, 3, None, 0, C.byref(info), None) == -1
    assert C.sizeof(Q.GesvdInfo) == 56


def test_struct_offsets_match_c_compiler(tmp_path):
    """sizeof and offsetof of every struct the binding mirrors, from gcc on the header."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_2104_14186_gb300 import qdwhp as Q
    structs = {"qdwhp_opts": Q.Opts, "qdwhp_info": Q.Info, "qdwhp_syev_info": Q.SyevInfo,
               "qdwhp_gesvd_info": Q.GesvdInfo}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "qdwhp.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                               text=True).stdout.split("\n") if line)
    for cname, py in structs.items():
        assert int(got[cname]) == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)


def test_tuning_table_checks_and_roundtrip(lib, tmp_path):
    """Launch-shape knobs: range checks, get/set/reset, and the autotuner's JSON table."""
    from paper_2104_14186_gb300 import autotune
    try:
        assert [lib.qdwhp_tune_get(k, 2) for k in range(3)] == [64, 2, 2]
        assert lib.qdwhp_tune_set(0, 2, 128) == 0 and lib.qdwhp_tune_get(0, 2) == 128
        assert lib.qdwhp_tune_set(0, 2, 8) == -1          # below the panel's 16 rows per CTA
        assert lib.qdwhp_tune_set(0, 2, 1024) == -1       # panel shared memory would pass 128 KB
        assert lib.qdwhp_tune_set(1, 0, 17) == -1
        assert lib.qdwhp_tune_set(2, 5, 2) == -1 and lib.qdwhp_tune_get(3, 0) == -1
        res = {"version": 1, "classes": [], "table": {"panel_rows_per_cta": [32, 64, 64, 128, 256],
                                                       "jacobi_min_warps": [4, 2, 2, 1, 1],
                                                       "splitk_ctas_per_sm": [2, 2, 4, 1, 2]}}
        path = str(tmp_path / "tune.json")
        autotune.save(res, path)
        got = autotune.load(path)
        assert got["table"] == res["table"]
        autotune.apply(got)
        assert lib.qdwhp_tune_get(0, 4) == 256 and lib.qdwhp_tune_get(1, 0) == 4 and lib.qdwhp_tune_get(2, 2) == 4
        bad = dict(res, table=dict(res["table"], jacobi_min_warps=[4, 2]))
        autotune.save(bad, path)
        with pytest.raises(ValueError):
            autotune.load(path)
    finally:
        lib.qdwhp_tune_reset()
    assert [lib.qdwhp_tune_get(k, 4) for k in range(3)] == [64, 2, 2]


def test_autotuner_coordinate_descent_on_a_known_cost(monkeypatch):
    """The tuner's search logic on the host, with the library and the timing replaced by a
    known cost: per class and knob it must keep the candidate of least cost, knob by knob."""
    from paper_2104_14186_gb300 import autotune

    table = {(k, c): v for k in range(3) for c in range(5) for v in [(64, 2, 2)[k]]}

    class FakeLib:
        def qdwhp_tune_get(self, k, c):
            return table[(k, c)]

        def qdwhp_tune_set(self, k, c, v):
            lo, hi = [(16, 512), (1, 16), (1, 8)][k]
            if not lo <= v <= hi:
                return -1
            table[(k, c)] = v
            return 0

    class FakeQ:
        @staticmethod
        def lib():
            return FakeLib()

    best = {0: {0: 128, 1: 32, 2: 256, 3: 64}, 1: {0: 4, 1: 1, 2: 8, 3: 2}, 2: {0: 1, 1: 4, 2: 2, 3: 4}}

    def cost(c):
        # separable cost, minimal at `best`; the tuner must find it one knob at a time
        return sum(abs(np.log2(table[(k, c)]) - np.log2(best[k][c])) for k in range(3)) + 1.0

    import numpy as np
    import sys
    from paper_2104_14186_gb300 import inputs
    monkeypatch.setattr(inputs, "eig_uniform_device", lambda n, seed, frac: (n, None, 1))
    monkeypatch.setattr(autotune, "_time_solve", lambda Q, A, k, reps: cost(autotune.CLASS_ORDERS.index(A)))
    import paper_2104_14186_gb300 as pkg
    fake_build = type("FakeBuild", (), {"build": staticmethod(lambda: None)})
    for name, mod in (("build", fake_build), ("qdwhp", FakeQ)):
        monkeypatch.setattr(pkg, name, mod, raising=False)
        monkeypatch.setitem(sys.modules, f"paper_2104_14186_gb300.{name}", mod)
    res = autotune.tune(classes=(0, 1, 2, 3), reps=1)
    for name, (k, _) in autotune.KNOBS.items():
        for c in range(4):
            assert res["table"][name][c] == best[k][c], (name, c, res["table"][name])
        assert res["table"][name][4] == (64, 2, 2)[k]     # class 4 untouched


def test_info_dict_slices_schedule_by_iterations(lib):
    """ell_k / conv hold one entry per polar iteration: QDWH steps (it_qr + it_chol) or, with
    Zolo-PD, its iterations (it_qr and it_chol then count terms)."""
    from paper_2104_14186_gb300 import qdwhp as Q
    info = Q.Info()
    info.it_qr, info.it_chol = 1, 5
    for i in range(12):
        info.ell_k[i] = 0.5 + i
    assert len(info.as_dict()["ell_k"]) == 6
    info.zolo_steps = 2
    d = info.as_dict()
    assert d["ell_k"] == [0.5, 1.5] and len(d["conv"]) == 2 and d["zolo_steps"] == 2
    g = Q.GesvdInfo()
    g.median_splits = 3
    assert g.as_dict()["median_splits"] == 3 and "reserved" not in g.as_dict()


def test_host_entry_points_argument_checks(lib):
    """The host-buffer forms size their workspace as the solver's plus the device copies of A
    and the outputs, and reject bad arguments before any copy or launch."""
    from paper_2104_14186_gb300 import qdwhp as Q
    o = Q.default_opts()
    o.count = 20
    eig_ws = lib.qdwhp_eig_workspace_bytes(300, C.byref(o))
    host_ws = lib.qdwhp_eig_host_workspace_bytes(300, C.byref(o))
    assert host_ws >= eig_ws + (300 * 300 + 20 + 300 * 20) * 8
    svd_ws = lib.qdwhp_svd_workspace_bytes(400, 300, C.byref(o))
    assert lib.qdwhp_svd_host_workspace_bytes(400, 300, 25, C.byref(o)) >= svd_ws + (400 * 300 + 25 * 701) * 8
    assert lib.qdwhp_svd_host_workspace_bytes(400, 300, 301, C.byref(o)) == 0     # k > min(m, n)
    assert lib.qdwhp_eig_host_workspace_bytes(0, C.byref(o)) == 0
    info = Q.Info()
    buf = (C.c_double * 16)()
    assert lib.qdwhp_eig_host(None, 300, 300, C.byref(o), buf, buf, 300, None, 0, C.byref(info), None) == -1
    assert lib.qdwhp_eig_host(buf, 300, 299, C.byref(o), buf, buf, 300, None, 0, C.byref(info), None) == -1
    assert lib.qdwhp_eig_host(buf, 300, 300, C.byref(o), buf, buf, 300, None, 0, C.byref(info), None) == -2
    assert lib.qdwhp_svd_host(buf, 400, 300, 400, 25, C.byref(o), buf, buf, 399, buf, 300, None, 0,
                              C.byref(info), None) == -1
    o.use_omega = 3
    assert lib.qdwhp_svd_host(buf, 400, 300, 400, 25, C.byref(o), buf, buf, 400, buf, 300, None, 0,
                              C.byref(info), None) == -1
