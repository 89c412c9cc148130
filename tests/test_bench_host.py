"""Host-side pieces of bench.py that the GPU run depends on: the clock sampler's parsing
(median SM clock under load, throttle reasons) and the peak lookup's fallback."""
import json

import bench


class _DoneProcess:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _sampler_with(tmp_path, lines):
    c = bench.Clocks(0)
    f = open(tmp_path / "clocks.csv", "w+")
    f.write("".join(line + "\n" for line in lines))
    f.flush()
    c.proc, c.file = _DoneProcess(), f
    return c


def test_clock_sampler_median_under_load_and_reasons(tmp_path):
    busy = "0, 2070, 2070, 1100.5, 0x4, Not Active, Not Active, Not Active, Active"
    idle = "0, 345, 2070, 120.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    out = _sampler_with(tmp_path, [idle, busy, busy, "0, 2055, 2070, 1090.0, 0x0, Not Active, Not Active, "
                                                     "Not Active, Not Active", idle]).stop()
    assert out["samples"] == 5
    assert out["sm_mhz"] == 2070.0            # idle samples (below half the peak) are left out
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert bench.clocks_sm_mhz(out) == 2070.0


def test_clock_sampler_reports_thermal_slowdown(tmp_path):
    hot = "0, 1800, 2070, 1300.0, 0x40, Not Active, Active, Not Active, Not Active"
    out = _sampler_with(tmp_path, [hot, hot]).stop()
    assert out["reasons"] == ["hw_thermal_slowdown"] and out["sm_mhz"] == 1800.0


def test_clock_sampler_without_nvidia_smi():
    out = bench.Clocks(0).stop()               # never started: no samples, no clock
    assert out["samples"] == 0 and out["sm_mhz"] is None
    assert bench.clocks_sm_mhz(out) is None


def test_peaks_measured_and_fallback(tmp_path, monkeypatch):
    p = tmp_path / "peaks.json"
    p.write_text(json.dumps({"hbm_gbs": 6686.8, "bf16_tflops": 1921.5}))
    monkeypatch.setattr(bench, "PEAKS_FILE", str(p))
    assert bench._peaks() == (6686.8, "measured")
    monkeypatch.setattr(bench, "PEAKS_FILE", str(tmp_path / "absent.json"))
    assert bench._peaks() == (bench.FALLBACK_HBM_GBS, "fallback")
