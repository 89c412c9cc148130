"""Pins of the oracle's STFT front end (Section 2), binary mask (the conclusion's future work)
and energy-weighted DOA error (Section 4, Eq. 16-20) against facts the paper and the
mathematics fix, each independent of the oracle's own code."""
import numpy as np
import pytest

import oracle as O
from oracle import frontend as F
from paper_1811_11785_gb300 import inputs as I


def _signal(M=3, S=1100, seed=1):
    return np.random.default_rng(seed).standard_normal((M, S))


def test_stft_equals_numpy_rfft_of_windowed_frames():
    x = _signal()
    N, hop = 128, 64
    X = F.stft(x, N, hop)
    w = F.sine_window(N)
    L = F.n_frames(x.shape[1], N, hop)
    assert X.shape == (L, 3, N // 2 + 1) and L == (1100 - 128) // 64 + 1
    for l in (0, 5, L - 1):
        ref = np.fft.rfft(x[:, l * hop:l * hop + N] * w, axis=1)
        assert np.max(np.abs(X[l] - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_stft_parseval_over_half_spectrum():
    x = _signal(M=2, S=512)
    N = 256
    X = F.stft(x, N, 128)
    w = F.sine_window(N)
    c = np.full(N // 2 + 1, 2.0)
    c[0] = c[-1] = 1.0
    for l in range(X.shape[0]):
        e_time = N * np.sum((x[:, l * 128:l * 128 + N] * w) ** 2, axis=1)
        e_freq = np.sum(c * np.abs(X[l]) ** 2, axis=1)
        assert np.allclose(e_freq, e_time, rtol=1e-12)


def test_sine_window_dc_closed_form():
    """A constant signal: X[0] = sum_n sin(pi (n + 1/2) / N) = 1 / sin(pi / (2N))."""
    for N in (8, 64, 512):
        X = F.stft(np.ones((1, N)), N, N)
        assert X[0, 0, 0].real == pytest.approx(1.0 / np.sin(np.pi / (2 * N)), rel=1e-12)
        assert abs(X[0, 0, 0].imag) < 1e-12


def test_impulse_fixes_window_hop_and_sign():
    """An impulse at sample s0 gives, in every frame l that holds it, X[k] = w[n0] exp(-2 pi i
    k n0 / N) with n0 = s0 - l hop: pins the window values, the frame offsets and the sign."""
    N, hop, s0 = 32, 8, 45
    x = np.zeros((1, 120))
    x[0, s0] = 1.0
    X = F.stft(x, N, hop)
    n = np.arange(N)
    w = np.sin(np.pi * (n + 0.5) / N)
    k = np.arange(N // 2 + 1)
    for l in range(X.shape[0]):
        n0 = s0 - l * hop
        if 0 <= n0 < N:
            assert np.allclose(X[l, 0], w[n0] * np.exp(-2j * np.pi * k * n0 / N), atol=1e-13)
        else:
            assert np.all(X[l, 0] == 0)


def test_mask_zeroes_bins_and_their_cross_spectra():
    x = _signal(M=3, S=300)
    N, hop = 64, 32
    L = F.n_frames(300, N, hop)
    mask = I.random_mask(np.random.default_rng(2), L, N // 2 + 1, 0.6)
    X = F.stft(x, N, hop)
    Xm = F.stft(x, N, hop, mask=mask)
    keep = mask.astype(bool)
    assert np.array_equal(Xm[:, :, ~keep[0]][0], np.zeros_like(Xm[:, :, ~keep[0]][0]))
    assert np.array_equal(Xm * 1, X * keep[:, None, :])
    assert np.array_equal(F.apply_mask(X, mask), Xm)
    P = O.phat(Xm).reshape(L, 3, N // 2 + 1)          # 3 pairs for 3 microphones
    assert np.all(P[~np.broadcast_to(keep[:, None, :], P.shape)] == 0)


def test_time_signals_carry_the_plane_wave_delay():
    """With no noise, the STFT cross spectra of the generated signals have the phase of Eq. 3-4
    for the source direction: a far-field source from u gives X_ij = conj(W_q(u)) per bin."""
    rng = np.random.default_rng(4)
    mic = I.array_3d()
    u = np.array([0.3, -0.5, 0.81])
    u /= np.linalg.norm(u)
    x = I.time_signals(rng, mic, 4096, 16000.0, 343.0, u, 200.0)
    N = 512
    X = F.stft(x.astype(np.float64), N, 256)
    tau = O.tdoa_farfield(mic, u[None, :], 16000.0, 343.0)
    W = O.steering(tau, N)
    Y = O.srp_scores(W, O.phat(X))
    L = W.shape[1]
    # the windowed-frame phase of a circularly delayed signal matches the ramp up to the window
    # edges; most of the energy is aligned
    assert np.all(Y[:, 0] > 0.9 * L)


def test_doa_maps_eq16_to_eq19():
    s = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.6, 0.0, -0.8]])
    f1 = F.doa_map(s, 1)
    g = np.arctan2(-0.8, 0.6)
    assert np.allclose(f1[3], [np.cos(g), 0, np.sin(g)])
    assert np.allclose(f1[:3], [[0, 0, 1], [1, 0, 0], [1, 0, 0]], atol=1e-12)
    assert np.allclose(F.doa_map(np.array([1.0, 2.0, -3.0]), 2), [1, 2, 3])
    assert np.array_equal(F.doa_map(s, 3), s)


def test_weighted_rmse_eq20():
    s0 = np.array([0.0, 0.0, 1.0])
    assert F.rmse_weighted(np.tile(s0, (5, 1)), np.arange(1, 6), s0, 3) == 0.0
    a, b = np.array([1.0, 0, 0]), np.array([0.0, 1.0, 0])
    # weights 1 and 3: mean = (a + 3 b) / 4 = (0.25, 0.75, 0)
    got = F.rmse_weighted(np.stack([a, b]), np.array([1.0, 3.0]), s0, 3)
    assert got == pytest.approx(np.sqrt(0.25 ** 2 + 0.75 ** 2 + 1.0), rel=1e-14)
    # the planar map folds the lower hemisphere: a mirrored estimate has no error
    assert F.rmse_weighted(np.array([[0.6, 0.0, -0.8]]), np.array([2.0]), np.array([0.6, 0.0, 0.8]), 2) == 0.0


def test_image_sources_first_order_and_gains():
    """The direct path and the six first-order images of a shoebox, with one coefficient each."""
    room = (10.0, 8.0, 3.0)
    beta = (0.1, 0.2, 0.3, 0.4, 0.5, 0.6)
    pos, g = I.image_sources([1.0, 2.0, 1.5], room, beta, 1)
    got = {tuple(np.round(p, 9)): gg for p, gg in zip(pos, g)}
    want = {(1.0, 2.0, 1.5): 1.0, (-1.0, 2.0, 1.5): 0.1, (19.0, 2.0, 1.5): 0.2, (1.0, -2.0, 1.5): 0.3,
            (1.0, 14.0, 1.5): 0.4, (1.0, 2.0, -1.5): 0.5, (1.0, 2.0, 4.5): 0.6}
    assert set(got) == set(want)
    for k, v in want.items():
        assert got[k] == pytest.approx(v)
    assert len(I.image_sources([1.0, 2.0, 1.5], room, beta, 2)[0]) == 25


def test_rir_direct_path_delay_and_gain():
    """Order 0: one windowed sinc at d fs / c with peak 1 / (4 pi d) for an integer delay."""
    fs, c = 16000.0, 343.0
    d = 343.0 * 100 / 16000.0                     # exactly 100 samples
    mic = np.array([[d, 0.0, 0.0]])
    h = I.room_impulse_responses(mic, np.zeros((1, 3)), np.ones(1), fs, c, 200)
    assert np.argmax(np.abs(h[0])) == 100
    assert h[0, 100] == pytest.approx(1.0 / (4 * np.pi * d), rel=1e-12)
    assert np.all(np.abs(np.delete(h[0], 100)) < 1e-12)
