"""Parity of the STFT front end (Section 2), the binary time-frequency mask (the paper's
conclusion) and localisation from time samples (Algorithm 1 from the samples on) with the FP64
oracle, through the C ABI.

Tolerance of the FP32 STFT against the FP64 DFT sum, per frame and channel: an FFT's rounding
error in 2-norm is at most a small multiple of u log2(N) ||X||_2 with ||X||_2 = sqrt(N) ||w x||_2
(Parseval over the full spectrum), so every bin is within 8 u log2(N) sqrt(N) ||w x||_2,
u = 2^-24."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1811_11785_gb300 as sp
from oracle import frontend as F
from paper_1811_11785_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _build():
    import __graft_entry__
    __graft_entry__.build()


def _stft_bound(x, N, hop, T):
    w = F.sine_window(N)
    nrm = np.array([[np.linalg.norm(w * x[m, l * hop:l * hop + N]) for m in range(x.shape[0])] for l in range(T)])
    return 8 * np.log2(N) * 2.0 ** -24 * np.sqrt(N) * nrm


@pytest.mark.parametrize("N,hop", [(8, 4), (64, 16), (512, 256), (1024, 512), (256, 3)])
def test_stft_matches_the_fp64_dft(N, hop):
    _build()
    rng = np.random.default_rng(N + hop)
    x = rng.standard_normal((7, 6 * N + 5)).astype(np.float32)
    Xg = sp.stft(torch.from_numpy(x).cuda(), N, hop).cpu().numpy()
    Xo = F.stft(x.astype(np.float64), N, hop)
    assert Xg.shape == Xo.shape and Xg.shape[0] == F.n_frames(x.shape[1], N, hop)
    err = np.max(np.abs(Xg - Xo), axis=2)
    assert np.all(err <= _stft_bound(x.astype(np.float64), N, hop, Xg.shape[0]))


def test_stft_short_signal_and_odd_row_stride():
    _build()
    x = torch.randn(3, 100, device="cuda")
    assert sp.stft(x, 128, 64).shape == (0, 3, 65)            # fewer samples than one frame
    big = torch.randn(3, 1001, device="cuda")
    view = big[:, :997]                                         # rows 1001 floats apart
    Xg = sp.stft(view, 64, 32).cpu().numpy()
    Xo = F.stft(big[:, :997].cpu().numpy().astype(np.float64), 64, 32)
    assert np.all(np.max(np.abs(Xg - Xo), axis=2) <= _stft_bound(big[:, :997].cpu().numpy().astype(np.float64),
                                                                  64, 32, Xg.shape[0]))


def test_mask_zeroes_bins_exactly():
    _build()
    rng = np.random.default_rng(7)
    x = torch.from_numpy(rng.standard_normal((7, 4096)).astype(np.float32)).cuda()
    N, hop = 512, 256
    T = sp.n_frames(4096, N, hop)
    mask = torch.from_numpy(I.random_mask(rng, T, N // 2 + 1, 0.5)).cuda()
    full = sp.stft(x, N, hop)
    masked = sp.stft(x, N, hop, mask=mask)
    keep = mask.bool()[:, None, :]
    assert torch.equal(masked, torch.where(keep, full, torch.zeros_like(full)))
    assert torch.equal(sp.apply_mask(full, mask), masked)
    inplace = full.clone()
    sp.apply_mask(inplace, mask, out=inplace)
    assert torch.equal(inplace, masked)


_W = {}


def _workload():
    """7-microphone planar array (Table 2 circle), one white source per segment of 16384
    samples (eight directions), white noise at 10 dB, N = 512, hop 256 (511 frames), Q = 642."""
    if "w" not in _W:
        _build()
        rng = np.random.default_rng(I.SEED_BASE + 70)
        mic = I.array_planar_2d_circle()
        segs = [I.time_signals(rng, mic, 16384, 16000.0, 343.0, u, 10.0) for u in I.random_directions(rng, 8)]
        x = np.concatenate(segs, axis=1)
        dirs = I.icosphere(3)
        st = sp.build_steering(mic, dirs, 16000.0, 343.0, 512)
        b = sp.svd_reduce(st, 1e-5)
        tau = O.tdoa_farfield(mic, dirs, 16000.0, 343.0)
        ob = O.svd_basis(O.steering(tau, 512), 1e-5)
        _W["w"] = dict(x=x, st=st, b=b, tau=tau, ob=ob, cls=O.direction_classes(tau),
                       xt=torch.from_numpy(x).cuda())
    return _W["w"]


def _agree(w, idx, Y):
    cls = w["cls"]
    ref, _ = O.argmax_lowest(Y)
    m = O.top2_margin(Y, cls)
    same = cls[idx] == cls[ref]
    assert np.all(same[m > 1e-4])
    assert len(idx) >= 400 and np.mean(same) >= 0.995
    return np.mean(same)


@pytest.mark.parametrize("prec", ["fp16", "fp32"])
def test_localize_samples_matches_stft_then_localize_and_the_oracle(prec):
    w = _workload()
    idx, score, proj = sp.localize_samples(w["b"], w["xt"], 256, "svd_exhaustive", prec)
    frames = sp.stft(w["xt"], 512, 256)
    i2, s2, p2 = sp.localize(w["b"], frames, "svd_exhaustive", prec)
    torch.cuda.synchronize()
    sp.check_status()
    assert torch.equal(idx, i2) and torch.equal(proj, p2) and torch.equal(score, s2)
    Xo = O.phat(F.stft(w["x"].astype(np.float64), 512, 256))
    Y = O.svd_scores(w["ob"]["D"], O.project(w["ob"]["V"], Xo))
    _agree(w, idx.cpu().numpy(), Y)
    L = w["st"].L
    sref = O.score_row(w["tau"], idx.cpu().numpy(), Xo, 512)
    assert np.max(np.abs(score.cpu().numpy() - sref)) <= 1e-5 * L


def test_localize_samples_with_a_mask():
    """Masked bins drop out of every score: the GPU path on masked samples equals the GPU path
    on masked STFT frames, and agrees with the oracle on masked frames (Eq. 3 zero rule)."""
    w = _workload()
    T = sp.n_frames(w["x"].shape[1], 512, 256)
    mask_np = I.random_mask(np.random.default_rng(9), T, 257, 0.7)
    mask = torch.from_numpy(mask_np).cuda()
    idx, score, proj = sp.localize_samples(w["b"], w["xt"], 256, "svd_exhaustive", "fp16", mask=mask)
    mf = sp.apply_mask(sp.stft(w["xt"], 512, 256), mask)
    i2, s2, p2 = sp.localize(w["b"], mf, "svd_exhaustive", "fp16")
    torch.cuda.synchronize()
    assert torch.equal(idx, i2) and torch.equal(proj, p2) and torch.equal(score, s2)
    Xo = O.phat(F.stft(w["x"].astype(np.float64), 512, 256, mask=mask_np))
    Y = O.svd_scores(w["ob"]["D"], O.project(w["ob"]["V"], Xo))
    _agree(w, idx.cpu().numpy(), Y)
    sref = O.score_row(w["tau"], idx.cpu().numpy(), Xo, 512)
    assert np.max(np.abs(score.cpu().numpy() - sref)) <= 1e-5 * w["st"].L
    # the masked bins are gone from the score: at most the kept bins' share of L
    assert np.all(score.cpu().numpy() <= mask_np.sum(axis=1) * w["st"].P * (1 + 1e-5))


def test_localize_samples_rejects_more_frames_than_the_samples_hold():
    w = _workload()
    T = sp.n_frames(w["x"].shape[1], 512, 256)
    with pytest.raises(sp.SvdPhatError):
        sp.localize_samples(w["b"], w["xt"], 256, T=T + 1)
