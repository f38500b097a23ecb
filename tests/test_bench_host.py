"""Host-side logic of the benchmark on CPU: the clock record built from
nvidia-smi samples (median under load, throttle reasons), the roofline
denominator read from the measured-peaks file, the CPU-baseline and CPU SpMV
records and the solution-error report."""
import json

import pytest

import bench


class _FakeProc:
    def __init__(self, text):
        self.text = text

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.text, ""


def _stop(text):
    s = bench.ClockSampler(0)
    s.proc = _FakeProc(text)
    return s.stop()


def _row(sm, smax=2070, reasons=("Not Active",) * 4, active="0x0"):
    return ", ".join(["0", str(sm), str(smax), "900.0", active, *reasons])


def test_clocks_median_is_taken_under_load():
    # idle samples (below half the highest clock) do not pull the median down
    rows = [_row(345), _row(345), _row(2070), _row(2040), _row(1980)]
    c = _stop("\n".join(rows))
    assert c["sm_mhz"] == 2040 and c["sm_max_mhz"] == 2070 and c["samples"] == 5 and c["reasons"] == []


def test_clocks_report_each_active_reason_once():
    pc = ("Not Active", "Not Active", "Not Active", "Active")
    th = ("Not Active", "Active", "Not Active", "Not Active")
    c = _stop("\n".join([_row(1900, reasons=pc), _row(1800, reasons=pc), _row(1700, reasons=th)]))
    assert c["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clocks_skip_malformed_lines():
    c = _stop("\n".join(["garbage", "0, [N/A], 2070, 1, 0x0, a, b, c, d", _row(2000)]))
    assert c["samples"] == 1 and c["sm_mhz"] == 2000


def test_clocks_without_samples_or_tool():
    assert _stop("")["reasons"] == ["no samples"]
    s = bench.ClockSampler(0)
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_peaks_reads_the_measured_copy_bandwidth(tmp_path, monkeypatch):
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6500.5}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6500.5, "measured")
    (tmp_path / "MEASURED_PEAKS.json").unlink()
    assert bench.peaks() == (6800.0, "fallback")


def test_cpu_baseline_is_the_full_jacobian_measurement():
    # measured on the benchmark's own 128x128x64 Jacobian: no scaling
    rec = bench.cpu_baseline_record(9.25, {"iters": 20})
    assert rec["value"] == pytest.approx(9.25e3)
    assert rec["unit"] == "ms" and rec["cores"] == 1 and rec["kind"] == "oracle"
    assert "20 its" in rec["sample"] and "128x128x64" in rec["sample"]
    assert rec["host_cores"] >= rec["affinity_cores"] >= 1


def test_solution_errors_overall_and_per_component():
    import numpy as np
    xr = np.array([1000.0, 0.2, 0.05] * 4)
    x = xr.copy()
    x[0::3] *= 1 + 1e-7
    x[2::3] *= 1 - 2e-6
    e = bench.solution_errors(x, xr)
    assert e["p"] == pytest.approx(1e-7, rel=1e-6) and e["sw"] == 0.0
    assert e["sg"] == pytest.approx(2e-6, rel=1e-6)
    assert e["all"] == pytest.approx(np.linalg.norm(x - xr) / np.linalg.norm(xr))


def test_cpu_spmv_record_counts_algorithmic_bytes():
    import bogen
    a = bogen.assemble(bogen.tiny_case(0))
    rec = bench.cpu_spmv_record(a, threads=2, reps=2)
    nnzb = bench._nnzb(20, 20, 5)
    assert rec["algorithmic_bytes"] == 72 * nnzb + 2 * 6000 * 8 and rec["gbs"] > 0 and rec["threads"] == 2
