"""Host-side bookkeeping of bench.py that decides whether a measurement is
kept: the clock record of the timed region, the roofline denominator and the
algorithmic flop count.  No GPU is involved."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _sampler(lines):
    s = bench.ClockSampler()
    s.lines = list(lines)
    return s


def test_clock_summary_median_and_reasons():
    na, act = "Not Active", "Active"
    lines = [
        f"2032, 2032, 905.1, {na}, {na}, {na}, {act}",
        f"1980, 2032, 1090.0, {na}, {na}, {na}, {na}",
        f"2010, 2032, 1010.3, {na}, {na}, {na}, {act}",
        "garbled line",
        f"[N/A], 2032, 1000.0, {na}, {na}, {na}, {na}",
    ]
    out = _sampler(lines).summary()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2010.0
    assert out["sm_max_mhz"] == 2032.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_summary_reports_each_slowdown_reason():
    na, act = "Not Active", "Active"
    out = _sampler([f"1500, 2032, 700.0, {act}, {act}, {act}, {na}"]).summary()
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    out = _sampler([]).summary()
    assert out == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}


def test_tensor_peak_prefers_sustained_then_burst_then_fallback(tmp_path):
    p = tmp_path / "MEASURED_PEAKS.json"
    assert bench.tensor_peak(str(tmp_path)) == (1400.0, "fallback bf16 sustained")
    p.write_text(json.dumps({"hbm_gbs": 7100.0, "bf16_tflops": 1790.0,
                             "bf16_tflops_sustained": 1401.0}))
    assert bench.tensor_peak(str(tmp_path)) == (1401.0, "measured bf16 sustained")
    p.write_text(json.dumps({"hbm_gbs": 7100.0, "bf16_tflops": 1790.0}))
    assert bench.tensor_peak(str(tmp_path)) == (1790.0, "measured bf16 burst")
    for bad in ('{"hbm_gbs": 7100.0}', "[1, 2]", "not json", '{"bf16_tflops_sustained": null}',
                '{"bf16_tflops_sustained": true}', '{"bf16_tflops_sustained": -1}'):
        p.write_text(bad)
        assert bench.tensor_peak(str(tmp_path)) == (1400.0, "fallback bf16 sustained")


@pytest.mark.parametrize("n_mu,rows,n_g", [(2000, 100000, 100000), (96, 17, 4800)])
def test_w_flops_counts_both_stages(n_mu, rows, n_g):
    # stage 1: 4 channels x one MAC per (nu, g, g'); stage 2: 4 channels x
    # one MAC per (mu, nu, g)
    s1 = 4 * 2 * n_mu * rows * n_g
    s2 = 4 * 2 * n_mu * n_mu * rows
    assert bench.w_flops(n_mu, rows, n_g) == s1 + s2
