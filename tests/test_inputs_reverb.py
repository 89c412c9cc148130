"""The seeded reverberant frame generator (input plumbing for the learned proposal's
training sets): plane-wave phases, the energy of the exponential tail, the SNR, and
reproducibility.  Runs on the CPU with torch's generator."""
import numpy as np
import pytest
import torch

from paper_1811_11785_gb300 import inputs as I

FS, C, N = 16000.0, 343.0, 256


def _mic():
    return I.array_random_ball(np.random.default_rng(3), 6)


def test_direct_path_is_a_plane_wave():
    mic = _mic()
    fr, dirs, ns = I.reverberant_frames_gpu(5, mic, 8, N, FS, C, max_sources=1, n_reflections=0,
                                            snr_range=(300.0, 300.0), device="cpu")
    k = np.arange(N // 2 + 1)
    for t in range(8):
        d = FS / C * (mic @ dirs[t, 0].numpy())
        ratio = fr[t].numpy().astype(np.complex128) / fr[t, 0].numpy()[None, :]
        want = np.exp(2j * np.pi * (d[:, None] - d[0]) * k[None, :] / N)
        assert np.max(np.abs(ratio - want)) < 1e-4
    assert torch.all(ns == 1)


@pytest.mark.parametrize("t60", [0.2, 0.6])
def test_tail_energy_follows_the_decay(t60):
    """Mean tail energy over direct energy = density * T60 / 13.8 (60 dB over T60)."""
    mic = _mic()
    args = dict(max_sources=1, snr_range=(300.0, 300.0), t60_range=(t60, t60), device="cpu")
    T = 4000
    dry, _, _ = I.reverberant_frames_gpu(7, mic, T, N, FS, C, n_reflections=0, **args)
    wet, _, _ = I.reverberant_frames_gpu(7, mic, T, N, FS, C, **args)
    e_dry = float((dry.abs() ** 2).mean())
    e_wet = float((wet.abs() ** 2).mean())
    want = I.REVERB_DENSITY * t60 * (1 - 1e-6) / (6 * np.log(10))
    assert abs((e_wet - e_dry) / e_dry - want) < 0.08 * want


def test_snr_and_source_counts():
    mic = _mic()
    fr, _, ns = I.reverberant_frames_gpu(9, mic, 3000, N, FS, C, snr_range=(0.0, 0.0), device="cpu")
    clean, _, _ = I.reverberant_frames_gpu(9, mic, 3000, N, FS, C, snr_range=(300.0, 300.0), device="cpu")
    ps = float((clean.abs() ** 2).mean())
    pn = float(((fr - clean).abs() ** 2).mean())
    assert abs(10 * np.log10(ps / pn)) < 0.2
    counts = np.bincount(ns.numpy(), minlength=4)[1:]
    assert np.all(np.abs(counts / 3000 - 1 / 3) < 0.04)


def test_seeded():
    mic = _mic()
    a = I.reverberant_frames_gpu(11, mic, 50, N, FS, C, device="cpu")
    b = I.reverberant_frames_gpu(11, mic, 50, N, FS, C, device="cpu")
    c = I.reverberant_frames_gpu(12, mic, 50, N, FS, C, device="cpu")
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])
    assert not torch.equal(a[0], c[0])
