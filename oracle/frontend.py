"""FP64 ORACLE for the parts around the SVD-PHAT hot path -- test infrastructure, NOT the product.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline`` /
``--impl reference`` legs import this module; the product library never does, and nothing
here imports the product.

* The STFT front end of Section 2: frames of N samples with hop Delta N, a sine window, and
  bins k = 0 .. N/2 (the expression X_m^l[k] that Eq. 3 starts from).
* The binary time-frequency mask the paper's conclusion proposes: a masked bin of a frame is
  a zero spectrum entry, so by the |X|^2 < 1e-30 rule of Eq. 3 every cross spectrum of that
  bin is 0 and the bin drops out of Eq. 5, 9, 12 and 14.
* The energy-weighted DOA error of Section 4 (Eq. 16-20) used for the delta sweep.

Readings of the paper:

* "sine window" is taken as w[n] = sin(pi (n + 1/2) / N), n = 0 .. N-1 (the paper names the
  window but prints no formula).
* The STFT is X_m^l[k] = sum_n w[n] x_m[l Delta N + n] exp(-2 pi i k n / N) with no
  normalisation (PHAT divides every entry by its magnitude, so a scale drops out).
* Frames: l = 0 .. floor((S - N) / Delta N) for S samples per channel (no padding).
* Eq. 20: Y_q in the weights is the SRP-PHAT energy of the chosen direction, Y_qbar of
  Algorithm 1's online step 4 (the same quantity for SRP-PHAT and SVD-PHAT).
"""
from __future__ import annotations

import numpy as np


def sine_window(N: int) -> np.ndarray:
    """w[n] = sin(pi (n + 1/2) / N), n = 0 .. N-1 (Section 2's sine window)."""
    n = np.arange(N, dtype=np.float64)
    return np.sin(np.pi * (n + 0.5) / N)


def n_frames(n_samples: int, N: int, hop: int) -> int:
    """Number of whole frames of N samples with hop Delta N in n_samples samples."""
    return 0 if n_samples < N else (n_samples - N) // hop + 1


def stft(x: np.ndarray, N: int, hop: int, mask: np.ndarray | None = None) -> np.ndarray:
    """Section 2: X[l][m][k] = sum_n w[n] x[m][l hop + n] exp(-2 pi i k n / N), k = 0 .. N/2.

    ``x`` is ``[M][S]`` (channel rows).  The DFT is written out as its matrix (FP64), one
    frame at a time.  ``mask`` (``[L][N/2+1]``, nonzero = keep) zeroes the masked bins of
    every channel.  Returns ``[L][M][N/2+1]`` complex128.
    """
    x = np.asarray(x, dtype=np.float64)
    M, S = x.shape
    L = n_frames(S, N, hop)
    B = N // 2 + 1
    w = sine_window(N)
    n = np.arange(N, dtype=np.float64)
    k = np.arange(B, dtype=np.float64)
    F = np.exp(-2j * np.pi * np.outer(n, k) / N)      # [N][B]: the DFT restricted to k <= N/2
    out = np.empty((L, M, B), dtype=np.complex128)
    for l in range(L):
        seg = x[:, l * hop: l * hop + N] * w[None, :]
        out[l] = seg @ F
    if mask is not None:
        out *= (np.asarray(mask) != 0)[:, None, :]
    return out


def apply_mask(frames: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """The binary time-frequency mask on STFT frames ``[L][M][B]``: bins with mask 0 become 0."""
    return np.asarray(frames) * (np.asarray(mask) != 0)[:, None, :]


# --------------------------------------------------------------------------------------
# Section 4: the energy-weighted DOA error (Eq. 16-20)
# --------------------------------------------------------------------------------------

def doa_map(s: np.ndarray, alpha: int) -> np.ndarray:
    """f_alpha of Section 4 for directions ``s`` (``[..][3]``): alpha = 1 maps to the arc
    [cos g, 0, sin g] with g = atan2(s_z, sqrt(s_x^2 + s_y^2)) (Eq. 16, 17), alpha = 2 to the
    upper hemisphere [s_x, s_y, |s_z|] (Eq. 18), alpha = 3 is the identity (Eq. 19)."""
    s = np.asarray(s, dtype=np.float64)
    if alpha == 1:
        g = np.arctan2(s[..., 2], np.sqrt(s[..., 0] ** 2 + s[..., 1] ** 2))
        return np.stack([np.cos(g), np.zeros_like(g), np.sin(g)], axis=-1)
    if alpha == 2:
        return np.stack([s[..., 0], s[..., 1], np.abs(s[..., 2])], axis=-1)
    if alpha == 3:
        return s.copy()
    raise ValueError("alpha must be 1, 2 or 3")


def rmse_weighted(s_hat: np.ndarray, Y: np.ndarray, s0: np.ndarray, alpha: int) -> float:
    """Eq. 20: || sum_l f(s_qbar_l) Y_l / sum_l Y_l - f(s0) ||_2 over the frames l of one
    configuration, with s_hat the chosen directions ``[L][3]`` and Y their energies ``[L]``."""
    f = doa_map(s_hat, alpha)
    Y = np.asarray(Y, dtype=np.float64)
    mean = (f * Y[:, None]).sum(axis=0) / Y.sum()
    return float(np.linalg.norm(mean - doa_map(np.asarray(s0, dtype=np.float64), alpha)))
