"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the FP64 oracle.

This module holds no arithmetic of the localisation method itself (no TDOA table,
no PHAT, no steering matrix, no SVD, no scoring).  It only produces the things the
method takes as *inputs*:

* the candidate-direction grid (icosphere; SVD-PHAT Section 4 uses 2562 points on a
  recursively subdivided unit sphere),
* microphone array geometries (Table 2 of the paper, plus the exact-circle planar
  variant and random arrays inside a 10 cm sphere),
* STFT frames of white-noise plane-wave sources with additive white or diffuse noise
  (the paper's TIMIT / image-method rooms are replaced by this synthetic workload).

Every generator takes an explicit ``numpy.random.Generator`` so a seed fixes the data.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 181111785

# --------------------------------------------------------------------------------------
# Direction grid
# --------------------------------------------------------------------------------------

_PHI = (1.0 + 5.0 ** 0.5) / 2.0

_ICO_VERTS = np.array(
    [
        [-1, _PHI, 0], [1, _PHI, 0], [-1, -_PHI, 0], [1, -_PHI, 0],
        [0, -1, _PHI], [0, 1, _PHI], [0, -1, -_PHI], [0, 1, -_PHI],
        [_PHI, 0, -1], [_PHI, 0, 1], [-_PHI, 0, -1], [-_PHI, 0, 1],
    ],
    dtype=np.float64,
)

_ICO_FACES = [
    (0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
    (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
    (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
    (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1),
]


def icosphere(level: int) -> np.ndarray:
    """Unit directions of an icosahedron subdivided ``level`` times: 10*4**level + 2 points.

    Order: the 12 base vertices, then each subdivision appends the (deduplicated) edge
    midpoints in face-traversal order, projected back onto the unit sphere.  Levels
    3/4/5/6 give 642/2562/10242/40962 directions.
    """
    if level < 0:
        raise ValueError("level must be >= 0")
    verts = [v / np.linalg.norm(v) for v in _ICO_VERTS]
    faces = list(_ICO_FACES)
    for _ in range(level):
        mid: dict[tuple[int, int], int] = {}

        def midpoint(a: int, b: int) -> int:
            key = (a, b) if a < b else (b, a)
            idx = mid.get(key)
            if idx is None:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                idx = len(verts) - 1
                mid[key] = idx
            return idx

        new_faces = []
        for (a, b, c) in faces:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            new_faces += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = new_faces
    out = np.ascontiguousarray(np.array(verts, dtype=np.float64))
    assert out.shape[0] == 10 * 4 ** level + 2
    return out


def icosphere_level_for(Q: int) -> int:
    for lvl in range(0, 9):
        if 10 * 4 ** lvl + 2 == Q:
            return lvl
    raise ValueError(f"Q={Q} is not an icosphere size")


# --------------------------------------------------------------------------------------
# Microphone arrays (metres)
# --------------------------------------------------------------------------------------

def array_linear_1d() -> np.ndarray:
    """Table 2, 1-D column: 7 mics on the z axis at -5,-3.3,-1.7,0,1.7,3.3,5 cm."""
    z = np.array([-5.0, -3.3, -1.7, 0.0, 1.7, 3.3, 5.0]) / 100.0
    return np.stack([np.zeros(7), np.zeros(7), z], axis=1)


def array_planar_2d_table() -> np.ndarray:
    """Table 2, 2-D column, literal printed coordinates (4.3 cm rather than 5 sin 60)."""
    xy = [(0, 0), (5, 0), (2.5, 4.3), (-2.5, 4.3), (-5.0, 0), (-2.5, -4.3), (2.5, -4.3)]
    return np.array([[x / 100.0, y / 100.0, 0.0] for x, y in xy], dtype=np.float64)


def array_planar_2d_circle() -> np.ndarray:
    """Centre mic plus 6 mics on an exact 5 cm circle at 60 degree steps (z = 0)."""
    pts = [[0.0, 0.0, 0.0]]
    for i in range(6):
        a = np.deg2rad(60.0 * i)
        pts.append([0.05 * np.cos(a), 0.05 * np.sin(a), 0.0])
    return np.array(pts, dtype=np.float64)


def array_3d() -> np.ndarray:
    """Table 2, 3-D column: centre, then -x,+x,-y,+y,-z,+z at 5 cm."""
    p = [(0, 0, 0), (-5, 0, 0), (5, 0, 0), (0, -5, 0), (0, 5, 0), (0, 0, -5), (0, 0, 5)]
    return np.array(p, dtype=np.float64) / 100.0


def array_random_ball(rng: np.random.Generator, M: int, radius: float = 0.05,
                      min_sep: float = 0.01) -> np.ndarray:
    """M mics drawn uniformly in a ball (rejecting any closer than ``min_sep``)."""
    pts: list[np.ndarray] = []
    while len(pts) < M:
        p = rng.uniform(-radius, radius, size=3)
        if np.dot(p, p) > radius * radius:
            continue
        if all(np.linalg.norm(p - q) >= min_sep for q in pts):
            pts.append(p)
    return np.array(pts, dtype=np.float64)


# --------------------------------------------------------------------------------------
# Random directions and STFT frames
# --------------------------------------------------------------------------------------

def random_directions(rng: np.random.Generator, n: int) -> np.ndarray:
    """n directions uniform on the unit sphere."""
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def hann(N: int) -> np.ndarray:
    """Periodic Hann window of length N."""
    n = np.arange(N)
    return 0.5 - 0.5 * np.cos(2.0 * np.pi * n / N)


def _windowed_spectra(rng: np.random.Generator, shape: tuple, N: int, win: np.ndarray):
    x = rng.standard_normal(shape + (N,))
    return np.fft.rfft(x * win, axis=-1)


def isotropic_mixing(mic_xyz: np.ndarray, N: int, fs: float, c: float) -> np.ndarray:
    """Per bin k, a matrix A_k with A_k A_k^T equal to the spherically isotropic coherence
    Gamma_ij = sinc(2 f_k d_ij / c) (numpy's normalised sinc), f_k = k fs / N: the
    symmetric square root from the eigendecomposition (negative rounding eigenvalues
    clipped to 0).  Shape (B, M, M)."""
    mic_xyz = np.asarray(mic_xyz, dtype=np.float64)
    d = np.linalg.norm(mic_xyz[:, None, :] - mic_xyz[None, :, :], axis=2)
    B = N // 2 + 1
    out = np.empty((B, mic_xyz.shape[0], mic_xyz.shape[0]))
    for k in range(B):
        G = np.sinc(2.0 * (k * fs / N) * d / c)
        lam, U = np.linalg.eigh(G)
        out[k] = (U * np.sqrt(np.clip(lam, 0.0, None))) @ U.T
    return out


def plane_wave_frames(
    rng: np.random.Generator,
    mic_xyz: np.ndarray,
    T: int,
    N: int,
    fs: float,
    c: float,
    src_dirs: np.ndarray,
    snr_db: np.ndarray,
    noise: str = "white",
    n_diffuse: int = 128,
    dtype=np.complex64,
) -> np.ndarray:
    """STFT frames ``[T][M][N/2+1]`` of white plane-wave sources plus noise.

    ``src_dirs`` is ``(T, S, 3)`` (S simultaneous sources per frame, unit vectors) and
    ``snr_db`` is ``(T,)``.  Each source is white Gaussian noise, Hann-windowed and
    transformed with an N-point real FFT; microphone m receives it advanced by
    ``fs/c * r_m . u`` samples, applied as a phase ramp in frequency
    (a fractional delay).  Noise is independent white noise per microphone
    (``noise='white'``), the sum of ``n_diffuse`` uncorrelated white plane waves
    from uniformly random directions (``noise='diffuse'``), or a spherically isotropic
    field (``noise='isotropic'``: the limit of infinitely many such plane waves, drawn
    per bin with the coherence sin(w d_ij / c) / (w d_ij / c) between microphones i and j
    at distance d_ij).  SNR is the mic-averaged
    signal power over noise power of that frame.
    """
    mic_xyz = np.asarray(mic_xyz, dtype=np.float64)
    M = mic_xyz.shape[0]
    B = N // 2 + 1
    src_dirs = np.asarray(src_dirs, dtype=np.float64)
    if src_dirs.ndim == 2:
        src_dirs = src_dirs[:, None, :]
    S = src_dirs.shape[1]
    win = hann(N)
    k = np.arange(B, dtype=np.float64)
    out = np.empty((T, M, B), dtype=dtype)
    if noise == "isotropic":
        iso_mix = isotropic_mixing(mic_xyz, N, fs, c)
    chunk = 4096
    for t0 in range(0, T, chunk):
        t1 = min(T, t0 + chunk)
        n = t1 - t0
        sig = np.zeros((n, M, B), dtype=np.complex128)
        spec = _windowed_spectra(rng, (n, S), N, win)  # (n, S, B)
        for s in range(S):
            d = (fs / c) * (src_dirs[t0:t1, s, :] @ mic_xyz.T)  # (n, M) advance in samples
            ph = np.exp(2j * np.pi * d[:, :, None] * k[None, None, :] / N)
            sig += spec[:, s, None, :] * ph
        if noise == "white":
            nz = _windowed_spectra(rng, (n, M), N, win)
        elif noise == "diffuse":
            nz = np.zeros((n, M, B), dtype=np.complex128)
            dirs = random_directions(rng, n * n_diffuse).reshape(n, n_diffuse, 3)
            sp = _windowed_spectra(rng, (n, n_diffuse), N, win)
            for j in range(n_diffuse):
                d = (fs / c) * (dirs[:, j, :] @ mic_xyz.T)
                nz += sp[:, j, None, :] * np.exp(2j * np.pi * d[:, :, None] * k[None, None, :] / N)
        elif noise == "isotropic":
            nz = np.einsum("kmj,njk->nmk", iso_mix, _windowed_spectra(rng, (n, M), N, win))
        else:
            raise ValueError(noise)
        ps = np.mean(np.abs(sig) ** 2, axis=(1, 2))
        pn = np.mean(np.abs(nz) ** 2, axis=(1, 2))
        g = np.sqrt(ps / (pn * 10.0 ** (np.asarray(snr_db[t0:t1], dtype=np.float64) / 10.0)))
        out[t0:t1] = (sig + g[:, None, None] * nz).astype(dtype)
    return out


def spherical_wave_frames(rng: np.random.Generator, mic_xyz: np.ndarray, N: int, fs: float, c: float,
                          src_xyz: np.ndarray, snr_db: np.ndarray, dtype=np.complex64) -> np.ndarray:
    """STFT frames ``[T][M][N/2+1]`` of one white point source per frame at position
    ``src_xyz[t]`` (metres) plus independent white noise per microphone: microphone m
    receives the source delayed by its distance, ``fs/c * ||s - r_m||`` samples, applied as
    a phase ramp in frequency.  SNR as in ``plane_wave_frames``."""
    mic_xyz = np.asarray(mic_xyz, dtype=np.float64)
    src_xyz = np.asarray(src_xyz, dtype=np.float64)
    T, M, B = src_xyz.shape[0], mic_xyz.shape[0], N // 2 + 1
    win = hann(N)
    k = np.arange(B, dtype=np.float64)
    spec = _windowed_spectra(rng, (T, 1), N, win)[:, 0, :]                          # (T, B)
    dist = np.sqrt(((src_xyz[:, None, :] - mic_xyz[None, :, :]) ** 2).sum(-1))       # (T, M)
    sig = spec[:, None, :] * np.exp(-2j * np.pi * (fs / c) * dist[:, :, None] * k[None, None, :] / N)
    nz = _windowed_spectra(rng, (T, M), N, win)
    ps = np.mean(np.abs(sig) ** 2, axis=(1, 2))
    pn = np.mean(np.abs(nz) ** 2, axis=(1, 2))
    g = np.sqrt(ps / (pn * 10.0 ** (np.asarray(snr_db, dtype=np.float64) / 10.0)))
    return (sig + g[:, None, None] * nz).astype(dtype)


def nearfield_points(level: int = 2, radii=(0.25, 0.5, 1.0)) -> np.ndarray:
    """Candidate source positions for the near-field steering (Eq. 1): the level-``level``
    icosphere directions at each radius (metres), radius-major."""
    u = icosphere(level)
    return np.concatenate([r * u for r in radii], axis=0)


# --------------------------------------------------------------------------------------
# Workload presets (the five configurations the build is measured on)
# --------------------------------------------------------------------------------------

def workload(name: str, T: int | None = None, seed_offset: int = 0):
    """Return a dict describing a preset workload and its seeded frames.

    Keys: mic_xyz, dirs (grid), fs, c, N, delta, frames [T][M][B] complex64,
    src_dirs (T,S,3), snr_db (T,).
    """
    fs, c = 16000.0, 343.0
    if name == "linear_q642":           # 7-mic line, Q=642, 100 frames, one direction, 10 dB
        rng = np.random.default_rng(SEED_BASE + 0 + seed_offset)
        mic, lvl, N = array_linear_1d(), 3, 512
        T = 100 if T is None else T
        u = random_directions(rng, 1)
        src = np.repeat(u[None, :, :], T, axis=0)
        snr = np.full(T, 10.0)
        frames = plane_wave_frames(rng, mic, T, N, fs, c, src, snr, "white")
    elif name == "planar_q2562":        # 7-mic planar circle, Q=2562, SNR U(-5,20)
        rng = np.random.default_rng(SEED_BASE + 1 + seed_offset)
        mic, lvl, N = array_planar_2d_circle(), 4, 512
        T = 65536 if T is None else T
        src = random_directions(rng, T)[:, None, :]
        snr = rng.uniform(-5.0, 20.0, size=T)
        frames = plane_wave_frames(rng, mic, T, N, fs, c, src, snr, "white")
    elif name == "array3d_q10242":      # 7-mic 3-D, Q=10242, 1-2 sources, isotropic noise 0-20 dB
        rng = np.random.default_rng(SEED_BASE + 3 + seed_offset)
        mic, lvl, N = array_3d(), 5, 512
        T = 1 << 20 if T is None else T
        S = 2
        src = random_directions(rng, T * S).reshape(T, S, 3)
        nsrc = rng.integers(1, 3, size=T)
        # a frame with one source gets its second source at zero amplitude: emulate by
        # duplicating the first direction (coherent sum keeps a single plane wave).
        src[nsrc == 1, 1, :] = src[nsrc == 1, 0, :]
        snr = rng.uniform(0.0, 20.0, size=T)
        frames = plane_wave_frames(rng, mic, T, N, fs, c, src, snr, "isotropic")
    elif name == "ball12_q642":         # 12 mics in a 5 cm-radius ball, Q=642, N=512: a wide basis
        rng = np.random.default_rng([SEED_BASE + 7, 1])
        mic, lvl, N = array_random_ball(rng, 12), 3, 512
        T = 300 if T is None else T
        src = random_directions(rng, T)[:, None, :]
        snr = rng.uniform(-5.0, 20.0, size=T)
        frames = plane_wave_frames(rng, mic, T, N, fs, c, src, snr, "white")
    elif name == "ball16_n1024_q642":   # 16 mics in a 5 cm-radius ball, N=1024, Q=642: 2K > 256
        rng = np.random.default_rng([SEED_BASE + 7, 4])
        mic, lvl, N = array_random_ball(rng, 16), 3, 1024
        T = 200 if T is None else T
        src = random_directions(rng, T)[:, None, :]
        snr = rng.uniform(-5.0, 20.0, size=T)
        frames = plane_wave_frames(rng, mic, T, N, fs, c, src, snr, "white")
    else:
        raise ValueError(f"unknown workload {name}")
    return dict(name=name, mic_xyz=mic, dirs=icosphere(lvl), fs=fs, c=c, N=N, delta=1e-5,
                frames=frames, src_dirs=src, snr_db=snr)


# --------------------------------------------------------------------------------------
# Learned proposal: seeded parameters and training frames
# --------------------------------------------------------------------------------------

def mlp_params(rng: np.random.Generator, F: int, H1: int, H2: int, C: int) -> np.ndarray:
    """A flat float32 parameter vector W1 [H1][F], b1, W2 [H2][H1], b2, W3 [C][H2], b3 with
    weights drawn N(0, 2 / fan_in) and biases N(0, 0.05^2)."""
    parts = []
    for rows, cols in ((H1, F), (H2, H1), (C, H2)):
        parts.append(rng.normal(0.0, np.sqrt(2.0 / cols), size=rows * cols))
        parts.append(rng.normal(0.0, 0.05, size=rows))
    return np.concatenate(parts).astype(np.float32)


def training_frames(rng: np.random.Generator, mic_xyz: np.ndarray, T: int, N: int, fs: float, c: float,
                    max_sources: int = 3, snr_range=(-5.0, 20.0)):
    """T frames with 1..max_sources white plane-wave sources from uniform random directions
    (a frame with fewer sources repeats its first direction), independent white noise at
    a uniform random SNR.  Returns (frames, src_dirs (T, S, 3), n_sources (T,))."""
    S = max_sources
    src = random_directions(rng, T * S).reshape(T, S, 3)
    ns = rng.integers(1, S + 1, size=T)
    for s in range(1, S):
        src[ns <= s, s, :] = src[ns <= s, 0, :]
    snr = rng.uniform(snr_range[0], snr_range[1], size=T)
    return plane_wave_frames(rng, mic_xyz, T, N, fs, c, src, snr, "white"), src, ns


# --------------------------------------------------------------------------------------
# Batched form: many independent streams
# --------------------------------------------------------------------------------------

def batched_streams(n: int, M_range=(4, 16), Q_choices=(642, 2562, 10242), N_choices=(256, 512, 1024),
                    T_range=(50, 2000), snr_range=(-5.0, 20.0), seed_offset: int = 0):
    """n streams, stream s drawn from its own generator keyed by (base seed + 2, s): M mics
    uniform in a 5 cm-radius ball (>= 1 cm apart), Q from Q_choices, N from N_choices, T
    uniform in T_range, one white plane-wave source per frame from a random direction, white
    noise at a per-stream SNR uniform in snr_range.  fs 16 kHz, c 343 m/s, delta 1e-5."""
    out = []
    for s in range(n):
        rng = np.random.default_rng([SEED_BASE + 2 + seed_offset, s])
        M = int(rng.integers(M_range[0], M_range[1] + 1))
        mic = array_random_ball(rng, M)
        Q = int(rng.choice(Q_choices))
        N = int(rng.choice(N_choices))
        T = int(rng.integers(T_range[0], T_range[1] + 1))
        snr = float(rng.uniform(*snr_range))
        src = random_directions(rng, T)[:, None, :]
        frames = plane_wave_frames(rng, mic, T, N, 16000.0, 343.0, src, np.full(T, snr), "white")
        out.append(dict(mic_xyz=mic, dirs=icosphere(icosphere_level_for(Q)), N=N, fs=16000.0, c=343.0,
                        delta=1e-5, frames=frames, src_dirs=src, snr_db=snr))
    return out


# --------------------------------------------------------------------------------------
# Time-domain signals for the STFT front end
# --------------------------------------------------------------------------------------

def time_signals(rng: np.random.Generator, mic_xyz: np.ndarray, S: int, fs: float, c: float,
                 src_dir: np.ndarray, snr_db: float) -> np.ndarray:
    """``[M][S]`` float32 samples: one white Gaussian source from direction ``src_dir`` (unit
    vector), microphone m receiving it advanced by fs/c r_m . u samples (a fractional, circular
    delay applied as a phase ramp over the whole signal's FFT), plus independent white noise at
    ``snr_db`` (microphone-averaged signal power over noise power)."""
    mic_xyz = np.asarray(mic_xyz, dtype=np.float64)
    u = np.asarray(src_dir, dtype=np.float64)
    u = u / np.linalg.norm(u)
    s = rng.standard_normal(S)
    Sf = np.fft.rfft(s)
    k = np.arange(Sf.shape[0])
    d = fs / c * (mic_xyz @ u)                       # advance of each microphone in samples
    x = np.fft.irfft(Sf[None, :] * np.exp(2j * np.pi * k[None, :] * d[:, None] / S), n=S, axis=1)
    p_sig = np.mean(x ** 2)
    noise = rng.standard_normal(x.shape) * np.sqrt(p_sig / 10.0 ** (snr_db / 10.0))
    return (x + noise).astype(np.float32)


def random_mask(rng: np.random.Generator, T: int, B: int, keep: float) -> np.ndarray:
    """A binary time-frequency mask ``[T][B]`` (uint8, 1 = keep) with each bin kept with
    probability ``keep``."""
    return (rng.random((T, B)) < keep).astype(np.uint8)


# --------------------------------------------------------------------------------------
# Synthetic shoebox rooms (the stand-in for Section 4's simulated rooms; TIMIT speech is not
# available, so the source is white noise)
# --------------------------------------------------------------------------------------

def image_sources(src, room, beta, order):
    """Image sources of a point source in a shoebox room [0, Lx] x [0, Ly] x [0, Lz] (the image
    method of Allen and Berkley, 1979): for every axis, image index n and parity p give the
    coordinate (1 - 2p) s + 2 n L, reflected |n - p| times on the wall at 0 and |n| times on the
    wall at L.  beta = (b_x0, b_xL, b_y0, b_yL, b_z0, b_zL) are the walls' reflection
    coefficients; images with more than `order` reflections in total are left out.  Returns
    (positions [I][3], gains [I]) with the gains the product of the coefficients."""
    src = np.asarray(src, dtype=np.float64)
    pos, gain = [], []
    rng_n = range(-order, order + 1)
    for nx in rng_n:
        for px in (0, 1):
            rx0, rxL = abs(nx - px), abs(nx)
            for ny in rng_n:
                for py in (0, 1):
                    ry0, ryL = abs(ny - py), abs(ny)
                    for nz in rng_n:
                        for pz in (0, 1):
                            rz0, rzL = abs(nz - pz), abs(nz)
                            if rx0 + rxL + ry0 + ryL + rz0 + rzL > order:
                                continue
                            pos.append([(1 - 2 * px) * src[0] + 2 * nx * room[0],
                                        (1 - 2 * py) * src[1] + 2 * ny * room[1],
                                        (1 - 2 * pz) * src[2] + 2 * nz * room[2]])
                            gain.append(beta[0] ** rx0 * beta[1] ** rxL * beta[2] ** ry0 * beta[3] ** ryL *
                                        beta[4] ** rz0 * beta[5] ** rzL)
    return np.array(pos), np.array(gain)


def room_impulse_responses(mic_pos, img_pos, img_gain, fs, c, length, half_width=16):
    """RIRs [M][length]: every image contributes gain / (4 pi d) at the fractional delay
    d fs / c samples, as a Hann-windowed sinc of 2 half_width + 1 taps."""
    M = mic_pos.shape[0]
    h = np.zeros((M, length))
    taps = np.arange(-half_width, half_width + 1)
    for m in range(M):
        d = np.linalg.norm(img_pos - mic_pos[m][None, :], axis=1)
        tau = d * fs / c
        amp = img_gain / (4.0 * np.pi * d)
        for t, a in zip(tau, amp):
            n0 = int(np.floor(t))
            idx = n0 + taps
            ok = (idx >= 0) & (idx < length)
            if not np.any(ok):
                continue
            x = idx - t
            w = 0.5 + 0.5 * np.cos(np.pi * x / (half_width + 1))
            h[m, idx[ok]] += a * (np.sinc(x) * w)[ok]
    return h


def room_signals(rng: np.random.Generator, mic_local: np.ndarray, S: int, fs: float, c: float,
                 room=(10.0, 10.0, 3.0), beta_range=(0.2, 0.5), snr_range=(0.0, 30.0), order: int = 2,
                 margin: float = 0.5):
    """One room configuration: the array (mic_local around its centre) and a source placed
    uniformly in the room at least `margin` from the walls and 1 m apart, wall reflection
    coefficients uniform in beta_range, the image method to `order` reflections, a white
    Gaussian source convolved with the RIRs, and independent white noise per channel at an SNR
    uniform in snr_range (microphone-averaged).  Returns (samples [M][S] float32, s0 the unit
    direction from the array centre to the source, beta, snr_db)."""
    room = np.asarray(room, dtype=np.float64)
    mic_local = np.asarray(mic_local, dtype=np.float64)
    while True:
        centre = margin + rng.random(3) * (room - 2 * margin)
        src = margin + rng.random(3) * (room - 2 * margin)
        if np.linalg.norm(src - centre) >= 1.0:
            break
    beta = rng.uniform(beta_range[0], beta_range[1], size=6)
    snr = float(rng.uniform(*snr_range))
    mics = centre[None, :] + mic_local
    img, g = image_sources(src, room, beta, order)
    dmax = np.max(np.linalg.norm(img - centre[None, :], axis=1)) + 0.2
    length = int(np.ceil(dmax * fs / c)) + 40
    h = room_impulse_responses(mics, img, g, fs, c, length)
    s = rng.standard_normal(S + length)
    nfft = 1 << int(np.ceil(np.log2(S + 2 * length)))
    x = np.fft.irfft(np.fft.rfft(s, nfft)[None, :] * np.fft.rfft(h, nfft, axis=1), nfft, axis=1)[:, length:length + S]
    p = np.mean(x ** 2)
    x = x + rng.standard_normal(x.shape) * np.sqrt(p / 10.0 ** (snr / 10.0))
    u = (src - centre) / np.linalg.norm(src - centre)
    return x.astype(np.float32), u, beta, snr


# --------------------------------------------------------------------------------------
# Reverberant frames generated on the device (the learned proposal's 2M-frame training sets)
# --------------------------------------------------------------------------------------

REVERB_DENSITY = 23.0      # reverberant energy per second at the onset, relative to the direct path
REVERB_REFLECTIONS = 8     # reflections drawn per source and frame


def reverberant_frames_gpu(seed: int, mic_xyz: np.ndarray, T: int, N: int, fs: float, c: float,
                           max_sources: int = 3, snr_range=(-5.0, 20.0), t60_range=(0.2, 0.6),
                           n_reflections: int = REVERB_REFLECTIONS, density: float = REVERB_DENSITY,
                           device="cuda", chunk: int = 16384):
    """STFT frames ``[T][M][N/2+1]`` (complex64 on ``device``) drawn with torch's seeded
    generator: 1..max_sources white sources per frame from uniformly random directions, each
    with an exponentially decaying reverberant tail, plus independent white noise per
    microphone at SNR ~ U(snr_range) (mic-averaged, against the reverberant signal).

    A source's spectrum is white complex Gaussian; microphone m receives a plane wave from u
    advanced by fs/c r_m . u samples (a phase ramp over the bins).  Its tail is n_reflections
    plane waves from uniformly random directions arriving t_r ~ U(0, T60) after the direct
    path, T60 ~ U(t60_range); reflection r carries energy density * T60 / n_reflections *
    10^(-6 t_r / T60) of the direct path's (a Monte Carlo sample of an energy envelope that
    decays by 60 dB over T60, so the tail holds density * T60 / 13.8 of the direct energy:
    -4.8 dB at T60 = 0.2 s, 0 dB at 0.6 s).  A reflection arriving a frame length or more
    after the direct sound carries an earlier, uncorrelated stretch of a white source, so each
    reflection gets its own white spectrum.  Returns (frames, directions [T][max_sources][3],
    number of sources [T]); rows s >= n_sources of the directions are unused."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    mic = torch.as_tensor(np.asarray(mic_xyz, dtype=np.float64), device=device).float()
    M, B = mic.shape[0], N // 2 + 1
    kb = torch.arange(B, device=device, dtype=torch.float32)

    def uniform(*shape):
        return torch.rand(shape, generator=g, device=device, dtype=torch.float32)

    def white(n):
        re = torch.randn((n, 1, B), generator=g, device=device, dtype=torch.float32)
        im = torch.randn((n, 1, B), generator=g, device=device, dtype=torch.float32)
        return torch.complex(re, im) * np.float32(np.sqrt(0.5))

    def unit(n):
        v = torch.randn((n, 3), generator=g, device=device, dtype=torch.float32)
        return v / v.norm(dim=1, keepdim=True)

    def plane(u):   # (n, 3) -> (n, M, B): phase ramps of plane waves from u
        d = (fs / c) * (u @ mic.T)
        ph = (2.0 * np.pi / N) * d[:, :, None] * kb[None, None, :]
        return torch.polar(torch.ones_like(ph), ph)

    out = torch.empty((T, M, B), dtype=torch.complex64, device=device)
    dirs = torch.zeros((T, max_sources, 3), dtype=torch.float32, device=device)
    n_src = torch.randint(1, max_sources + 1, (T,), generator=g, device=device)
    for t0 in range(0, T, chunk):
        n = min(chunk, T - t0)
        sig = torch.zeros((n, M, B), dtype=torch.complex64, device=device)
        for s in range(max_sources):
            active = (n_src[t0:t0 + n] > s).float()[:, None, None]
            u = unit(n)
            dirs[t0:t0 + n, s] = u
            sig += active * white(n) * plane(u)
            t60 = t60_range[0] + (t60_range[1] - t60_range[0]) * uniform(n, 1, 1)
            for _ in range(n_reflections):
                tr = uniform(n, 1, 1) * t60
                amp = torch.sqrt(density * t60 / n_reflections * torch.pow(10.0, -6.0 * tr / t60))
                sig += (active * amp) * white(n) * plane(unit(n))
        ps = (sig.abs() ** 2).mean(dim=(1, 2))
        snr = snr_range[0] + (snr_range[1] - snr_range[0]) * uniform(n)
        re = torch.randn((n, M, B), generator=g, device=device, dtype=torch.float32)
        im = torch.randn((n, M, B), generator=g, device=device, dtype=torch.float32)
        scale = torch.sqrt(ps / (2.0 * torch.pow(10.0, snr / 10.0)))[:, None, None]
        out[t0:t0 + n] = sig + torch.complex(re, im) * scale
    return out, dirs.double(), n_src
