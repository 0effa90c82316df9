"""Host-side arithmetic of bench.py (no GPU): the derived ALU peaks the roofline is taken
against, the bound and fraction it reports from a kernel's algorithmic bytes, flops, launch
count and time, and the command line."""
import importlib.util
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_host_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_derived_alu_peaks():
    b = load_bench()
    # 152 SMs x 2 FP64 FMA lanes x 2 flop x 2.07 GHz; x 128 FP32 lanes; df64 at 7.5 FP32
    # instructions per flop
    assert abs(b.alu_peak_tflops("f64", 2070.0) - 152 * 2 * 2 * 2.07e9 / 1e12) < 1e-12
    assert abs(b.alu_peak_tflops("f32", 2070.0) - 152 * 128 * 2 * 2.07e9 / 1e12) < 1e-9
    assert abs(b.alu_peak_tflops("df64", 2070.0) - 152 * 128 * 2.07e9 / 7.5 / 1e12) < 1e-9


def test_roofline_bound_and_fraction():
    b = load_bench()
    pk = {"hbm_gbs": 6794.5, "sm_max_mhz": 2070.0}
    # streaming kernel: 1 GB and 0.01 GFLOP per launch, 10 launches in 2 ms -> 5000 GB/s
    d = {"launches": 10, "ms": 2.0, "bytes": 1e10, "flops": 1e8}
    r = b.roofline("cheby_update", 0, d, pk, "measured")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 5000.0) < 0.1 and abs(r["frac"] - 5000.0 / 6794.5) < 1e-4
    # FP64 operator at p = 7 (variant 7: p = 7, kind f64): 1.8623 GFLOP and 1.133 GB per 1.423 ms
    d = {"launches": 1, "ms": 1.423, "bytes": 1.133e9, "flops": 1.8623e9}
    r = b.roofline("ax", 7, d, pk, "measured")
    peak = 152 * 2 * 2 * 2.07e9 / 1e12
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["kernel"] == "ax p=7 f64"
    assert abs(r["achieved"] - 1.8623e9 / 1.423e-3 / 1e12) < 1e-3
    assert abs(r["frac"] - r["achieved"] / peak) < 1e-3
    # FP32 variant (32 + p): the FP32 roof applies
    r = b.roofline("fdm", 39, {"launches": 36, "ms": 5.4, "bytes": 36 * 2.4e8, "flops": 36 * 3.28e9},
                   pk, "measured")
    assert r["kernel"] == "fdm p=7 f32" and r["bound"] == "alu"


def test_command_line_parses():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"],
                         capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and "--smoother" in out.stdout and "--cycle" in out.stdout
    bad = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--cycle", "additive"],
                         capture_output=True, text=True, timeout=120)
    assert bad.returncode != 0 and "additive" in bad.stderr
