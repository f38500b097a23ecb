"""Host-side logic of the benchmark on CPU: the clock record built from
nvidia-smi samples (median under load, throttle reasons), the roofline
denominator read from the measured-peaks file, and the CPU-baseline record's
scaling from the oracle sample to the full workload."""
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


def test_cpu_baseline_scales_by_the_cell_ratio():
    rec = bench.cpu_baseline_record(1.5, {"iters": 17})
    ratio = (128 * 128 * 64) / (64 * 64 * 32)
    assert rec["value"] == pytest.approx(1.5e3 * ratio)
    assert rec["unit"] == "ms" and rec["cores"] == 1 and rec["kind"] == "oracle"
    assert "17 its" in rec["sample"] and "64x64x32" in rec["sample"]
