"""bench.py's host-side arithmetic (no GPU): the roofline entries, the
derived FP32 peak and the choice of the dominant kernel."""
import pytest

import bench

PEAKS = {"hbm_gbs": 6788.6, "sm_max_mhz": 2070.0}


def test_alu_peak_from_units_and_clock():
    assert bench.alu_peak(PEAKS) == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)


def test_hbm_and_alu_entries():
    e = bench.hbm_entry("k", 6.7886e9, 1e-3, 2, PEAKS, "measured", "bytes")
    assert e["achieved"] == pytest.approx(6788.6) and e["frac"] == pytest.approx(1.0)
    assert e["step_ms"] == pytest.approx(2.0) and e["bound"] == "hbm" and e["unit"] == "GB/s"
    a = bench.alu_entry("w", 80.54784e9, 1e-3, 1, PEAKS, "flops")
    assert a["frac"] == pytest.approx(1.0, rel=1e-6) and a["bound"] == "alu" and a["unit"] == "TFLOP/s"


def test_reconstruction_roofline_counts_phi_once_and_frames():
    n, r, K = 1000, 10, 50
    e = bench.roofline(n, r, K, 1e-3, "mixed", PEAKS, "measured")
    assert e["achieved"] == pytest.approx(4.0 * n * (r + K) / 1e-3 / 1e9)
    f = bench.roofline(n, r, K, 1e-3, "fp32", PEAKS, "measured")
    assert f["achieved"] == pytest.approx(2.0 * n * r * K / 1e-3 / 1e12)


def test_whole_job_rate_is_weak_scaling_aggregate():
    assert bench.whole_job_rate(1000.0, 0.5, 1) == pytest.approx(2000.0)
    assert bench.whole_job_rate(1000.0, 0.5, 4) == pytest.approx(8000.0)


def test_profiling_case_helpers_resolve():
    """Every helper the --case dispatcher calls is defined at module level."""
    import ast
    import os
    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py")).read()
    tree = ast.parse(src)
    defined = {n.name for n in tree.body if isinstance(n, ast.FunctionDef)}
    called = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.FunctionDef) and node.name in ("run_case", "_case_model"):
            for sub in ast.walk(node):
                if isinstance(sub, ast.Call) and isinstance(sub.func, ast.Name) and sub.func.id.startswith("_case"):
                    called.add(sub.func.id)
    assert called and called <= defined, called - defined
