"""FP64 ORACLE for the SVD-PHAT hot path -- test infrastructure, NOT the product.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline`` /
``--impl reference`` legs import this package.  The product library
(``paper_1811_11785_gb300``) never imports, links or executes anything here, and this
package imports nothing from the product: the two share no code.  The only common
module is ``paper_1811_11785_gb300.inputs`` (seeded synthetic inputs, which holds none of
the method's arithmetic); this package does not even import that.

Everything is plain FP64 (complex128) numpy written to be checked against the paper by
eye, in the paper's own layout and notation:

* pairs (i, j), i < j, in the order (1,2), (1,3), ..., (M-1, M)              (Eq. 7)
* column index of X / W is ``p * B + k`` with ``B = N/2 + 1`` bins k=0..N/2    (Eq. 7, 8)
* a library matmul / eigendecomposition may stand in for a plain sum; there is no
  blocking, fusion or reordering beyond what the equations state.

Readings of the paper (where it is silent, garbled or inconsistent):

* Eq. 14's ``Re{D_q . Z^H}`` is read as the unconjugated row-times-column product
  ``Re{sum_k D_qk Z_k}``: only that reading makes SVD-PHAT equal SRP-PHAT at full rank.
* Eq. 15 holds for the normalised vectors: ``Re{D^_q Z^} = 1 - 1/2 ||D^_q - conj(Z^)||^2``.
* Section 3's ``K_max = max{Q, P(N/2+1)}`` is read as ``min`` (the rank bound).
* A spectrum entry whose squared magnitude is below 1e-30 is "zero" and every cross
  spectrum that uses it is 0 (Eq. 3 divides by the magnitudes).
* Ties in an argmax go to the lowest index.
* Eq. 1 (near field) takes ``s_q`` as a candidate source position in the microphones'
  frame; Eq. 2 is its limit for a distant source (Section 2), pinned as such.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle_jacobi.so")
_lib = None
_lock = threading.Lock()

ZERO_MAG2 = 1e-30


def build_c() -> str:
    """Compile the oracle's C part (the Jacobi eigen-iteration) with plain -O2."""
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_HERE, "jacobi.c")
    if (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               src, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_c())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_jacobi_herm.argtypes = [ctypes.c_int, dp, dp, dp, dp,
                                               ctypes.c_double, ctypes.c_int]
            lib.oracle_jacobi_herm.restype = ctypes.c_int
            _lib = lib
    return _lib


# --------------------------------------------------------------------------------------
# Section 2: SRP-PHAT
# --------------------------------------------------------------------------------------

def pairs(M: int) -> list[tuple[int, int]]:
    """Microphone pairs (i, j), i < j, in the order of Eq. 7: (1,2), (1,3), ..., (M-1,M)."""
    return [(i, j) for i in range(M) for j in range(i + 1, M)]


def tdoa_farfield(mic_xyz, dirs, fs: float, c: float) -> np.ndarray:
    """Eq. 2 (far field): ``tau[q, p] = fs/c * (r_j - r_i) . s_q / ||s_q||`` in samples.

    Evaluation order is fixed so the table is reproducible to the last bit:
    ``n = sqrt((sx*sx + sy*sy) + sz*sz)``, ``u = s / n`` (per component),
    ``tau = (fs / c) * ((dx*ux + dy*uy) + dz*uz)`` with ``d = r_j - r_i``;
    every operation rounds to nearest, no fused multiply-add.
    """
    r = np.asarray(mic_xyz, dtype=np.float64)
    s = np.asarray(dirs, dtype=np.float64)
    n = np.sqrt((s[:, 0] * s[:, 0] + s[:, 1] * s[:, 1]) + s[:, 2] * s[:, 2])
    ux, uy, uz = s[:, 0] / n, s[:, 1] / n, s[:, 2] / n
    g = np.float64(fs) / np.float64(c)
    P = pairs(r.shape[0])
    tau = np.empty((s.shape[0], len(P)), dtype=np.float64)
    for p, (i, j) in enumerate(P):
        dx, dy, dz = r[j, 0] - r[i, 0], r[j, 1] - r[i, 1], r[j, 2] - r[i, 2]
        tau[:, p] = g * ((dx * ux + dy * uy) + dz * uz)
    return tau


def tdoa_nearfield(mic_xyz, src_xyz, fs: float, c: float) -> np.ndarray:
    """Eq. 1 (near field): ``tau[q, p] = fs/c * (||s_q - r_i|| - ||s_q - r_j||)`` in samples,
    for source positions ``s_q``.

    Evaluation order is fixed so the table is reproducible to the last bit:
    ``n_m = sqrt((ex*ex + ey*ey) + ez*ez)`` with ``e = s_q - r_m``, then
    ``tau = (fs / c) * (n_i - n_j)``; every operation rounds to nearest, no fused
    multiply-add.
    """
    r = np.asarray(mic_xyz, dtype=np.float64)
    s = np.asarray(src_xyz, dtype=np.float64)
    dist = np.empty((s.shape[0], r.shape[0]), dtype=np.float64)
    for m in range(r.shape[0]):
        ex, ey, ez = s[:, 0] - r[m, 0], s[:, 1] - r[m, 1], s[:, 2] - r[m, 2]
        dist[:, m] = np.sqrt((ex * ex + ey * ey) + ez * ez)
    g = np.float64(fs) / np.float64(c)
    P = pairs(r.shape[0])
    tau = np.empty((s.shape[0], len(P)), dtype=np.float64)
    for p, (i, j) in enumerate(P):
        tau[:, p] = g * (dist[:, i] - dist[:, j])
    return tau


def steering(tau: np.ndarray, N: int) -> np.ndarray:
    """Eq. 4 stacked as Eq. 8: ``W[q, p*B + k] = exp(2 pi i k tau[q,p] / N)``, k=0..N/2."""
    Q, P = tau.shape
    B = N // 2 + 1
    k = np.arange(B, dtype=np.float64)
    ph = 2.0 * np.pi * k[None, None, :] * tau[:, :, None] / N
    return np.exp(1j * ph).reshape(Q, P * B)


def phat(frames: np.ndarray) -> np.ndarray:
    """Eq. 3 stacked as Eq. 7: ``X[t, p*B + k] = X_i[k] conj(X_j[k]) / (|X_i[k]| |X_j[k]|)``.

    ``frames`` is ``[T][M][B]`` complex.  An entry with ``|X_m[k]|^2 < 1e-30`` counts as
    zero and every cross spectrum that uses it is 0.
    """
    F = np.asarray(frames).astype(np.complex128)
    T, M, B = F.shape
    P = pairs(M)
    mag2 = F.real * F.real + F.imag * F.imag
    zero = mag2 < ZERO_MAG2
    out = np.empty((T, len(P), B), dtype=np.complex128)
    for p, (i, j) in enumerate(P):
        num = F[:, i, :] * np.conj(F[:, j, :])
        den = np.abs(F[:, i, :]) * np.abs(F[:, j, :])
        bad = zero[:, i, :] | zero[:, j, :]
        out[:, p, :] = np.where(bad, 0.0, num / np.where(bad, 1.0, den))
    return out.reshape(T, len(P) * B)


def srp_scores(W: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Eq. 5 / Eq. 9: ``Y[t, q] = Re{ sum_l W[q, l] X[t, l] }`` (no conjugation)."""
    return (np.asarray(X) @ np.asarray(W).T).real


def argmax_lowest(Y: np.ndarray):
    """Eq. 6 / Eq. 14: index of the maximum of each row (ties -> lowest index) and its value."""
    idx = np.argmax(Y, axis=1)  # numpy returns the first maximum
    return idx.astype(np.int64), Y[np.arange(Y.shape[0]), idx]


# --------------------------------------------------------------------------------------
# Section 3: SVD-PHAT
# --------------------------------------------------------------------------------------

def jacobi_eigh(G: np.ndarray, tol: float = 1e-14, max_sweeps: int = 60):
    """Hermitian eigendecomposition by the cyclic complex Jacobi iteration (C code).

    Returns eigenvalues in descending order and the matching unit eigenvectors as columns.
    """
    lib = _load()
    G = np.asarray(G, dtype=np.complex128)
    n = G.shape[0]
    Ar = np.ascontiguousarray(G.real.copy())
    Ai = np.ascontiguousarray(G.imag.copy())
    Vr = np.empty((n, n))
    Vi = np.empty((n, n))
    dp = ctypes.POINTER(ctypes.c_double)
    sweeps = lib.oracle_jacobi_herm(n, Ar.ctypes.data_as(dp), Ai.ctypes.data_as(dp),
                                    Vr.ctypes.data_as(dp), Vi.ctypes.data_as(dp),
                                    float(tol), int(max_sweeps))
    if sweeps < 0:
        raise RuntimeError("Jacobi iteration did not converge")
    lam = np.diag(Ar).copy()
    order = np.argsort(-lam, kind="stable")
    return lam[order], (Vr + 1j * Vi).T[:, order]     # the C code returns the eigenvectors as rows


def lapack_eigh(G: np.ndarray):
    """Hermitian eigendecomposition by LAPACK (numpy), descending order."""
    lam, U = np.linalg.eigh(np.asarray(G, dtype=np.complex128))
    return lam[::-1].copy(), U[:, ::-1].copy()


JACOBI_MAX_N = 700


CLUSTER_TOL = 1e-10


def rank_from_delta(sigma2: np.ndarray, trace: float, delta: float,
                    close_clusters: bool = True) -> int:
    """Eq. 11: the smallest K with ``sum_{k<=K} sigma_k^2 >= (1 - delta) Tr{W W^H}``.

    Reading: when that K would split a cluster of equal singular values (symmetric
    arrays give exact multiplets), the rank-K subspace -- and hence every SVD-PHAT score --
    is not unique; K is then extended to the end of the cluster
    (``sigma_{K+1}^2 >= sigma_K^2 - 1e-10 sigma_1^2``).
    """
    s2 = np.asarray(sigma2, dtype=np.float64)
    cs = np.cumsum(s2)
    hit = np.nonzero(cs >= (1.0 - delta) * trace)[0]
    K = int(hit[0]) + 1 if hit.size else int(len(cs))
    if close_clusters:
        while K < len(s2) and s2[K] >= s2[K - 1] - CLUSTER_TOL * s2[0]:
            K += 1
    return K


def svd_basis(W: np.ndarray, delta: float, eig: str = "auto", K: int | None = None) -> dict:
    """Eq. 10-13 and Algorithm 1 (offline steps 2-3).

    Truncated SVD ``W ~= U S V^H`` via the Gram matrix of W's smaller side:
    ``W W^H = U S^2 U^H`` (Q <= L) or ``W^H W = V S^2 V^H`` (Q > L).  K is chosen by Eq. 11
    (or given), ``V`` is ``L x K`` (``V = W^H U S^-1`` in the first case), ``D = U S = W V``
    (Eq. 13) and ``Dhat`` holds the unit-norm rows ``D_q / ||D_q||`` (Section 3).

    ``eig``: 'jacobi' (the oracle's own cyclic Jacobi), 'lapack' (numpy's eigh), or 'auto'
    (Jacobi up to n = 700, which covers every Q = 642 grid in about ten seconds, LAPACK above,
    where the Jacobi sweeps take minutes).
    """
    W = np.asarray(W, dtype=np.complex128)
    Q, L = W.shape
    trace = float(np.sum(W.real * W.real + W.imag * W.imag))  # Tr{W W^H}
    small_q = Q <= L
    G = W @ W.conj().T if small_q else W.conj().T @ W
    n = G.shape[0]
    if eig == "auto":
        eig = "jacobi" if n <= JACOBI_MAX_N else "lapack"
    lam, E = jacobi_eigh(G) if eig == "jacobi" else lapack_eigh(G)
    sigma2 = np.clip(lam, 0.0, None)
    if K is None:
        K = rank_from_delta(sigma2, trace, delta)
    K = int(K)
    if small_q:
        s = np.sqrt(sigma2[:K])
        V = (W.conj().T @ E[:, :K]) / s[None, :]
    else:
        V = E[:, :K].copy()
    D = W @ V
    nrm = np.sqrt(np.sum(D.real * D.real + D.imag * D.imag, axis=1))
    Dhat = D / nrm[:, None]
    return dict(K=K, sigma2=sigma2, trace=trace, V=V, D=D, Dhat=Dhat, eig=eig)


def project(V: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Eq. 12: ``Z = V^H X`` for every frame: ``Z[t, k] = sum_l conj(V[l, k]) X[t, l]``."""
    return np.asarray(X) @ np.asarray(V).conj()


def svd_scores(D: np.ndarray, Z: np.ndarray) -> np.ndarray:
    """Eq. 14: ``Y[t, q] = Re{ sum_k D[q, k] Z[t, k] }`` (unconjugated reading)."""
    return (np.asarray(Z) @ np.asarray(D).T).real


def nn_brute(Dhat: np.ndarray, Z: np.ndarray):
    """Eq. 15: nearest row of ``Dhat`` to ``conj(Z / ||Z||)`` (ties -> lowest index).

    Returns (index, squared distance) per frame; minimising this distance maximises
    ``Re{Dhat_q Zhat}``.
    """
    Z = np.asarray(Z, dtype=np.complex128)
    zn = np.sqrt(np.sum(Z.real * Z.real + Z.imag * Z.imag, axis=1))
    Zh = np.conj(Z / zn[:, None])
    out_i = np.empty(Z.shape[0], dtype=np.int64)
    out_d = np.empty(Z.shape[0])
    step = max(1, min(256, (1 << 23) // max(1, Dhat.size)))   # frames per block (memory only)
    for t0 in range(0, Z.shape[0], step):
        zz = Zh[t0:t0 + step]
        diff = Dhat[None, :, :] - zz[:, None, :]
        d2 = np.sum(diff.real * diff.real + diff.imag * diff.imag, axis=2)
        i = np.argmin(d2, axis=1)
        out_i[t0:t0 + step] = i
        out_d[t0:t0 + step] = d2[np.arange(len(i)), i]
    return out_i, out_d


def score_row(tau: np.ndarray, qbar, X: np.ndarray, N: int) -> np.ndarray:
    """Algorithm 1, online step 4: ``Y_qbar = Re{W_qbar X}`` with the row W_qbar of Eq. 8
    regenerated from the TDOA table."""
    qbar = np.asarray(qbar, dtype=np.int64)
    Wrows = steering(tau[qbar], N)  # (T, L)
    return np.sum((Wrows * np.asarray(X)).real, axis=1)


# --------------------------------------------------------------------------------------
# Helpers for comparing results (ties from array symmetry)
# --------------------------------------------------------------------------------------

def direction_classes(tau: np.ndarray, tol: float = 1e-9) -> np.ndarray:
    """Equivalence classes of directions with identical TDOA vectors (max |dtau| <= tol).

    Identical TDOA rows give identical rows of W, hence identical scores (a line array
    cannot tell directions on a cone apart, a planar array mirror images).  Returns, for
    every q, the lowest index of its class.
    """
    Q = tau.shape[0]
    cls = np.arange(Q)
    order = np.argsort(tau[:, 0], kind="stable")
    t0 = tau[order, 0]
    for a in range(Q):
        qa = order[a]
        b = a + 1
        while b < Q and t0[b] - t0[a] <= tol:
            qb = order[b]
            if np.max(np.abs(tau[qa] - tau[qb])) <= tol:
                lo = min(cls[qa], cls[qb])
                cls[qa] = cls[qb] = lo
            b += 1
    # propagate to the class minimum
    for _ in range(4):
        cls = cls[cls]
    return cls


def top2_margin(Y: np.ndarray, cls: np.ndarray) -> np.ndarray:
    """(Y1 - Y2) / |Y1| where Y2 is the best score outside the winning class."""
    idx = np.argmax(Y, axis=1)
    Y1 = Y[np.arange(Y.shape[0]), idx]
    same = cls[None, :] == cls[idx][:, None]
    Y2 = np.where(same, -np.inf, Y).max(axis=1)
    return (Y1 - Y2) / np.abs(Y1)
