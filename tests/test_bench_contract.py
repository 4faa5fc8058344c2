"""The reference arm of bench.py runs the oracle on the host (no GPU), so its JSON line can
be checked here: one solve of the 4096 x 4096 workload, the keys the bench contract names,
and the reference arm's own cpu_baseline and zero-copy e2e."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600, check=True).stdout
    line = json.loads(out.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["unit"] == "solves/s" and line["value"] > 0
    assert line["n_gpus"] == 1 and line["steps"] == 1 and line["higher_is_better"] is True
    assert line["config"]["workload"].startswith("QDWHpartial-SVD 4096x4096")
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert abs(line["ms_per_step"] - 1e3 / line["value"]) <= 1e-6 * line["ms_per_step"]


def test_reference_arm_under_two_ranks_prints_once():
    """Under torchrun with two ranks (gloo) rank 0 alone runs and prints; rank 1 exits 0."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0


def test_clock_summary_flags_throttle_reasons():
    """The clocks object of the bench line from nvidia-smi rows: median SM clock, max clock,
    the throttle reasons seen Active, unparsable rows skipped."""
    sys.path.insert(0, ROOT)
    import bench
    s = bench.ClockSampler(0)
    row = lambda sm, cap: [str(sm), "2070", "900.5", "0x0", "Not Active", "Not Active", "Not Active", cap]
    s.rows = [row(2070, "Not Active"), row(1980, "Active"), row(2070, "Not Active"),
              ["[N/A]", "[N/A]", "", "", "", "", "", ""]]
    out = s.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    s2 = bench.ClockSampler(0)
    s2.rows = [[str(1500), "2070", "1", "0x1", "Active", "Not Active", "Active", "Not Active"]]
    assert s2.stop()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_emulated_roofline_counts_algorithmic_flops():
    """The emulated-product roofline: 60 digit products of 2mnk (n(n+1)k for a lower SYRK)
    per recorded product, over the summed launch time, against the BF16 peak."""
    sys.path.insert(0, ROOT)
    import bench

    class FakeQ:
        @staticmethod
        def profile_records():
            # m, n, k, lower, split (-1: emulated), ms
            return [(4096.0, 4096.0, 4096.0, 0.0, -1.0, 10.0), (256.0, 256.0, 512.0, 1.0, -1.0, 0.5),
                    (512.0, 512.0, 512.0, 0.0, 1.0, 3.0)]    # a native DMMA record: ignored

    r = bench.emulated_roofline(FakeQ, 100.0, 2000.0)
    fp64 = 2.0 * 4096 ** 3 + 256 * 257 * 512
    assert r["launches"] == 2 and r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - 60 * fp64 / 10.5e-3 / 1e12) <= 1e-9 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / 2000.0) <= 1e-12
    assert abs(r["fp64_equivalent_tflops"] - fp64 / 10.5e-3 / 1e12) <= 1e-9 * r["fp64_equivalent_tflops"]
    assert abs(r["share_of_step"] - 10.5 / 100.0) <= 1e-12
