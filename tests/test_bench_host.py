"""Host-side arithmetic of bench.py's rooflines (no device involved)."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_alu_roofline_picks_the_binding_pipe():
    b = _bench()
    # 1 reciprocal + 6 binary32 per Voigt evaluation; MUFU 16 and FP32 128 lanes per SM per clock
    probe = {"fma_lane_ops_per_s": 128 * 100 * 1e9, "rcp_lane_ops_per_s": 16 * 100 * 1e9}
    r = b.alu_roofline(1.0e12, "voigt", probe, n_sm=100, clock_mhz=1000.0)
    assert r["pipe"] == "MUFU reciprocal"        # 1/16 > 6/128
    assert r["achieved"] == pytest.approx(1.0)    # 1e12 reciprocals/s
    assert r["peak"] == pytest.approx(1.6)
    assert r["frac"] == pytest.approx(1.0 / 1.6)
    assert r["other_pipe_frac"] == pytest.approx(6.0e12 / 12.8e12)
    assert r["derived_peaks_tops"] == pytest.approx({"fp32": 12.8, "mufu": 1.6})
    # an FP32-heavy mix (hypothetical slow FP32 pipe) binds on FP32
    slow = {"fma_lane_ops_per_s": 4e12, "rcp_lane_ops_per_s": 16e12}
    r2 = b.alu_roofline(0.5e12, "lorentz", slow, n_sm=100, clock_mhz=1000.0)
    assert r2["pipe"] == "FP32" and r2["frac"] == pytest.approx(0.5e12 * 4 / 4e12)
