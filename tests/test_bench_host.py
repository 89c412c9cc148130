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


def test_parallel_oracle_sample_matches_the_serial_oracle():
    """The CPU baseline splits the oracle's frames over spawned processes; the per-frame results
    (argmax and scores) are those of the oracle run in one process."""
    import numpy as np

    import oracle as O
    from paper_1811_11785_gb300 import inputs as I
    rng = np.random.default_rng(3)
    mic = I.array_3d()
    dirs = I.icosphere(2)
    src = I.random_directions(rng, 40)[:, None, :]
    fr = I.plane_wave_frames(rng, mic, 40, 64, 16000.0, 343.0, src, np.full(40, 10.0), "white")
    wl = dict(mic_xyz=mic, dirs=dirs, fs=16000.0, c=343.0, N=64, delta=1e-5, frames=fr)
    rate, dt, sel, idx, Y, cls = bench.oracle_sample(wl, 24, seed=5)
    assert rate > 0 and len(sel) == 24
    tau = O.tdoa_farfield(mic, dirs, 16000.0, 343.0)
    ob = O.svd_basis(O.steering(tau, 64), 1e-5)
    Yser = O.svd_scores(ob["D"], O.project(ob["V"], O.phat(fr[sel])))
    assert np.max(np.abs(Y - Yser)) <= 1e-9 * tau.shape[1] * 33
    assert np.array_equal(idx, O.argmax_lowest(Yser)[0])
    s4 = bench.oracle_step4(idx, 64)
    assert np.allclose(s4, O.score_row(tau, idx, O.phat(fr[sel]), 64), rtol=0, atol=1e-9)
