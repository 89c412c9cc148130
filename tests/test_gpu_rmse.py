"""Section 4's evaluation on the device: the energy-weighted DOA error (Eq. 16-20) against the
FP64 oracle, and a small delta sweep on synthetic shoebox rooms (image method, white-noise
sources): K falls as delta grows (Eq. 11) and at delta = 1e-5 SVD-PHAT's error is SRP-PHAT's."""
import numpy as np
import pytest
import torch

import paper_1811_11785_gb300 as sp
from oracle import frontend as F
from paper_1811_11785_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _build():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("alpha", [1, 2, 3])
def test_weighted_doa_error_matches_the_oracle(alpha):
    _build()
    rng = np.random.default_rng(30 + alpha)
    dirs = I.icosphere(3)
    st = sp.build_steering(I.array_3d(), dirs, 16000.0, 343.0, 64)
    T = 1000
    idx = rng.integers(0, len(dirs), size=T).astype(np.int32)
    Y = rng.uniform(0.5, 50.0, size=T).astype(np.float32)
    idx[7] = -1                      # frames the search could not score are left out
    Y[11] = np.nan
    s0 = np.array([0.2, -0.4, 0.9])
    got = sp.weighted_doa_error(st, torch.from_numpy(idx).cuda(), torch.from_numpy(Y).cuda(), s0, alpha)
    ok = (idx >= 0) & np.isfinite(Y)
    ref = F.rmse_weighted(dirs[idx[ok]] / np.linalg.norm(dirs[idx[ok]], axis=1, keepdims=True), Y[ok], s0 / np.linalg.norm(s0), alpha)
    assert got == pytest.approx(ref, rel=1e-12, abs=1e-14)


def test_small_delta_sweep_on_rooms():
    _build()
    fs, c, N, hop = 16000.0, 343.0, 256, 128
    dirs = I.icosphere(4)
    mic = I.array_3d()
    st = sp.build_steering(mic, dirs, fs, c, N, materialize_w=True)
    deltas = [1e-7, 1e-5, 1e-2]
    bases = [sp.svd_reduce(st, d) for d in deltas]
    Ks = [b.K for b in bases]
    assert Ks[0] >= Ks[1] >= Ks[2] and Ks[0] > Ks[2]
    rng = np.random.default_rng(I.SEED_BASE + 95)
    d_srp, d_svd = [], []
    for _ in range(4):
        x, s0, _, _ = I.room_signals(rng, mic, 12000, fs, c)
        frames = sp.stft(torch.from_numpy(x).cuda(), N, hop)
        i0, y0 = sp.localize_srp(st, frames)
        d_srp.append(sp.weighted_doa_error(st, i0, y0, s0, 3))
        i1, y1, _ = sp.localize(bases[1], frames, "svd_exhaustive", "fp32")
        d_svd.append(sp.weighted_doa_error(st, i1, y1, s0, 3))
    assert all(0 <= v <= 2 for v in d_srp + d_svd)
    assert abs(np.mean(d_svd) - np.mean(d_srp)) <= 0.05
