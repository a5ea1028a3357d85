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


def test_reference_arm_prints_one_contract_line():
    """bench.py --impl reference times the oracle on the host (no GPU) and
    prints one JSON line with the contract's keys; its cpu_baseline and e2e
    describe the same run, with no host-device copies."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "h6_chain", "--steps", "2", "--warmup", "1",
                        "--cpu-rows", "4"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["unit"] == "TFLOP/s" and line["value"] > 0
    assert line["steps"] == 2 and line["warmup"] == 1 and line["higher_is_better"] is True
    assert line["dtype"] == "f64" and line["config"]["workload"] == "h6_chain"
    assert line["config"]["l2"].startswith("inputs fit in L2")     # 4800 x 96: a small case
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    assert "4 of 4800 outer grid points" in cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
