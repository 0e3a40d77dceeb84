"""bench.py's reference arm (the FP64 oracle on the host cores) keeps the JSON-line contract:
one line with impl "reference", the metric, unit and direction of the GPU arm, a value that
equals its cpu_baseline and e2e values, and zero host/device bytes; and the roofline record
of the GPU arm picks the bound, the algorithmic figure and the peak of the dominant kernel
class.  Runs on the CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..")


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--workload", "wells2d-32"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["unit"] == "solves/s" and rec["higher_is_better"] is True
    assert rec["value"] > 0 and rec["steps"] == 1 and rec["warmup"] == 0
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["value"] == rec["value"]
    assert rec["e2e"] == {"value": rec["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}
    assert rec["config"]["workload"].startswith("wells2d-32")
    # the config states the refilter rounds the sample is scaled to (bench.py's default: 1)
    assert rec["config"]["refilter"] == 1 and "refilter_rtol" not in rec["config"]
    assert "rtol 1e-05" in rec["config"]["gmres"]


def test_roofline_record_bounds_and_arithmetic():
    """The dominant class's roofline: HBM bytes for the memory-bound classes; for the Gram
    class 48 n N^2 flops per call against FP32 FMA on the CUDA cores (152 SMs x 128 lanes x
    2 x clock) or, on tcgen05, the measured bf16 rate x 1.1 / 2.25."""
    import types
    import bench
    peaks = {"hbm_gbs": 6655.0, "bf16_tflops": 1937.4, "sm_max_mhz": 2070.0}
    prof = {"trsv_levels": {"calls": 10, "kernels": 10, "ms": 2.0, "bytes": 1.0e9, "impl_bytes": 3.0e9},
            "gram": {"calls": 4, "kernels": 8, "ms": 2.0, "bytes": 1.0e8}}
    wl = types.SimpleNamespace(N=128, n=16384)
    r = bench.roofline_record(prof, "trsv_levels", wl, peaks, 2070.0, 0, 5)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 500.0) < 1e-9 and abs(r["frac"] - 500.0 / 6655.0) < 1e-12
    # per call of the class: the algorithmic and the implementation's own bytes
    assert abs(r["algorithmic_bytes_per_call"] - 1.0e8) < 1e-3
    assert abs(r["impl_bytes_per_call"] - 3.0e8) < 1e-3
    assert "alu" not in r                      # no flops counted: no arithmetic sub-record
    # with the library's flop count of the supernode products: the same class against FP32 FMA
    prof["trsv_levels"]["flops"] = 4.0e10
    r = bench.roofline_record(prof, "trsv_levels", wl, peaks, 2070.0, 0, 5)
    assert r["bound"] == "hbm" and r["alu"]["unit"] == "TFLOP/s"
    assert abs(r["alu"]["achieved"] - 4.0e10 / 2.0e-3 / 1e12) < 1e-9
    assert abs(r["alu"]["peak"] - 152 * 128 * 2 * 2070e6 / 1e12) < 1e-9
    assert abs(r["alu"]["flops_per_call"] - 4.0e9) < 1e-3
    r = bench.roofline_record(prof, "gram", wl, peaks, 2000.0, 0, 5)
    flops = 4 * 48.0 * 16384 * 128 ** 2
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - flops / 2.0e-3 / 1e12) < 1e-9
    assert abs(r["peak"] - 152 * 128 * 2 * 2000e6 / 1e12) < 1e-9
    r = bench.roofline_record(prof, "gram", wl, peaks, None, 1, 5)
    assert r["bound"] == "tensor" and abs(r["peak"] - 1937.4 * 1.1 / 2.25) < 1e-9
