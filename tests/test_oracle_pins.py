"""Pins for the FP64 oracle: each test checks the oracle against something other than
itself -- values the paper prints, closed forms, textbook special cases, brute force on
tiny inputs and invariants the paper states -- so that a dropped term, a wrong sign or
index or a transposed operand in the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1811_11785_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _noiseless_frames(mic, u, T, N, fs, c, seed=0):
    rng = np.random.default_rng(seed)
    src = np.repeat(np.asarray(u, dtype=np.float64)[None, None, :], T, axis=0)
    # 400 dB SNR: the additive noise is ~1e-20 of the signal
    return I.plane_wave_frames(rng, mic, T, N, fs, c, src, np.full(T, 400.0), "white",
                               dtype=np.complex128)


# ---------------------------------------------------------------------------- pairs / TDOA

def test_pair_order_eq7():
    assert O.pairs(4) == [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    assert len(O.pairs(7)) == 21 and len(O.pairs(16)) == 120


def test_farfield_is_limit_of_nearfield_eq1_eq2():
    """Eq. 2 is the far-field limit of Eq. 1 (an independent formula): at 100 km the two
    agree to ~||r||^2/(2R) * fs/c samples; a sign or pair-order error would not."""
    mic = I.array_3d() + np.array([0.01, -0.02, 0.003])
    u = I.random_directions(np.random.default_rng(1), 50)
    far = O.tdoa_farfield(mic, u, 16000.0, 343.0)
    near = O.tdoa_nearfield(mic, 1e5 * u, 16000.0, 343.0)
    assert np.max(np.abs(far - near)) < 1e-5
    assert np.max(np.abs(far)) > 1.0


def test_tdoa_hand_value():
    """Two mics 8c/fs apart on x: a source on +x gives tau = fs/c (r_j - r_i).u = 8 samples."""
    c, fs = 343.0, 16000.0
    mic = np.array([[0.0, 0, 0], [8 * c / fs, 0, 0]])
    tau = O.tdoa_farfield(mic, np.array([[1.0, 0, 0], [0, 1.0, 0], [-2.0, 0, 0]]), fs, c)
    assert tau[:, 0] == pytest.approx([8.0, 0.0, -8.0], abs=1e-12)


def test_nearfield_tdoa_hand_values_eq1():
    """Eq. 1 by hand: two mics 8c/fs apart on x; a source on the axis beyond mic 1 is
    8 samples closer to it (tau = +8), beyond mic 0 the opposite (-8), on the perpendicular
    bisector 0; a source sitting on mic 0 gives -(fs/c) * ||r_1 - r_0|| = -8."""
    c, fs = 343.0, 16000.0
    a = 8 * c / fs
    mic = np.array([[0.0, 0, 0], [a, 0, 0]])
    src = np.array([[2.0, 0, 0], [-2.0, 0, 0], [a / 2, 1.3, -0.4], [0.0, 0, 0]])
    tau = O.tdoa_nearfield(mic, src, fs, c)
    assert tau[:, 0] == pytest.approx([8.0, -8.0, 0.0, -8.0], abs=1e-9)


def test_nearfield_tdoa_is_a_difference_of_distances():
    """Eq. 1 for every pair is d_j - d_i with d_m = -fs/c ||s - r_m||, so around any mic
    triangle the TDOAs close: tau_ij + tau_jk = tau_ik; and swapping a pair negates it."""
    rng = np.random.default_rng(3)
    mic = I.array_random_ball(rng, 6)
    src = rng.normal(size=(40, 3)) * 0.7
    tau = O.tdoa_nearfield(mic, src, 16000.0, 343.0)
    P = {pq: p for p, pq in enumerate(O.pairs(6))}
    for (i, j, k) in [(0, 1, 2), (1, 3, 5), (0, 2, 4), (2, 4, 5)]:
        assert np.max(np.abs(tau[:, P[(i, j)]] + tau[:, P[(j, k)]] - tau[:, P[(i, k)]])) < 1e-11
    flipped = O.tdoa_nearfield(mic[::-1], src, 16000.0, 343.0)
    assert np.max(np.abs(flipped[:, P[(0, 5)]] + tau[:, P[(0, 5)]])) < 1e-11   # pair (5, 0) reversed


def test_dirs_need_not_be_unit():
    mic = I.array_planar_2d_circle()
    u = I.icosphere(2)
    assert np.array_equal(O.tdoa_farfield(mic, u, 16000, 343), O.tdoa_farfield(mic, u * 1.0, 16000, 343))
    assert np.allclose(O.tdoa_farfield(mic, 3.7 * u, 16000, 343), O.tdoa_farfield(mic, u, 16000, 343),
                       atol=1e-13)


# ---------------------------------------------------------------------------- PHAT

def test_phat_unit_modulus_eq3():
    rng = np.random.default_rng(2)
    F = rng.standard_normal((5, 4, 33)) + 1j * rng.standard_normal((5, 4, 33))
    X = O.phat(F)
    assert X.shape == (5, 6 * 33)
    assert np.max(np.abs(np.abs(X) - 1.0)) < 1e-15


def test_phat_pair_layout_and_conjugate_eq3_eq7():
    """X[t, p*B + k] for pair p=(i,j) equals e^{i(arg X_i - arg X_j)} (checked on phases)."""
    rng = np.random.default_rng(3)
    ang = rng.uniform(-np.pi, np.pi, size=(2, 3, 5))
    F = rng.uniform(0.5, 2.0, size=(2, 3, 5)) * np.exp(1j * ang)
    X = O.phat(F).reshape(2, 3, 5)
    for p, (i, j) in enumerate([(0, 1), (0, 2), (1, 2)]):
        assert np.allclose(X[:, p, :], np.exp(1j * (ang[:, i, :] - ang[:, j, :])), atol=1e-14)


def test_phat_zero_entries_give_zero():
    F = np.ones((1, 3, 4), dtype=np.complex128)
    F[0, 1, 2] = 0.0
    X = O.phat(F).reshape(1, 3, 4)
    assert X[0, 0, 2] == 0 and X[0, 2, 2] == 0 and X[0, 1, 2] == 1.0
    assert np.all(np.abs(X[0, :, [0, 1, 3]]) == 1.0)


# ---------------------------------------------------------------------------- W and Gram

def test_steering_rows_have_equal_norm_and_trace_eq4_eq8():
    mic = I.array_planar_2d_table()
    tau = O.tdoa_farfield(mic, I.icosphere(2), 16000.0, 343.0)
    W = O.steering(tau, 64)
    L = 21 * 33
    assert W.shape == (162, L)
    assert np.allclose(np.sum(np.abs(W) ** 2, axis=1), L, atol=1e-10)
    assert np.sum(np.abs(W) ** 2) == pytest.approx(162 * L, rel=1e-14)
    assert np.allclose(W[:, 0::33], 1.0)  # k = 0 column of every pair


def test_gram_matches_dirichlet_closed_form():
    """G_{qq'} = sum_p sum_{k=0}^{B-1} e^{i 2 pi k (tau_qp - tau_q'p)/N}: a geometric series
    per pair, e^{i(B-1)th/2} sin(B th/2) / sin(th/2) with th = 2 pi dtau / N."""
    mic = I.array_3d()
    tau = O.tdoa_farfield(mic, I.icosphere(1), 16000.0, 343.0)
    N = 64
    B = N // 2 + 1
    W = O.steering(tau, N)
    G = W @ W.conj().T
    th = 2 * np.pi * (tau[:, None, :] - tau[None, :, :]) / N
    with np.errstate(invalid="ignore", divide="ignore"):
        term = np.exp(1j * (B - 1) * th / 2) * np.sin(B * th / 2) / np.sin(th / 2)
    term = np.where(np.abs(np.sin(th / 2)) < 1e-300, B, term)
    Gc = term.sum(axis=2)
    assert np.max(np.abs(G - Gc)) < 1e-9


# ---------------------------------------------------------------------------- SRP

def test_srp_brute_force_triple_sum_eq5():
    """Eq. 5 written out with explicit loops over i, j > i, k on a tiny case."""
    rng = np.random.default_rng(4)
    M, N, fs, c = 3, 8, 16000.0, 343.0
    B = N // 2 + 1
    mic = rng.uniform(-0.05, 0.05, size=(M, 3))
    dirs = I.icosphere(0)  # Q = 12
    F = rng.standard_normal((2, M, B)) + 1j * rng.standard_normal((2, M, B))
    Y = O.srp_scores(O.steering(O.tdoa_farfield(mic, dirs, fs, c), N), O.phat(F))
    for t in range(2):
        for q in range(12):
            u = dirs[q] / math.sqrt(float(dirs[q] @ dirs[q]))
            acc = 0j
            for i in range(M):
                for j in range(i + 1, M):
                    tau = fs / c * float((mic[j] - mic[i]) @ u)
                    for k in range(B):
                        xij = F[t, i, k] * np.conj(F[t, j, k]) / (abs(F[t, i, k]) * abs(F[t, j, k]))
                        acc += np.exp(2j * math.pi * k * tau / N) * xij
            assert Y[t, q] == pytest.approx(acc.real, abs=1e-12)


def test_m2_reduces_to_gcc_phat_at_integer_lags():
    """With M = 2 the SRP-PHAT score at an integer TDOA n is the GCC-PHAT value at lag n,
    obtained here from numpy's inverse real FFT: Y(n) = (N r[n] + X0 + X_{N/2} (-1)^n) / 2."""
    rng = np.random.default_rng(5)
    N, fs, c = 32, 16000.0, 343.0
    d = 8 * c / fs
    mic = np.array([[0.0, 0, 0], [d, 0, 0]])
    lags = np.arange(-8, 9)
    ux = lags / 8.0
    dirs = np.stack([ux, np.sqrt(1 - ux ** 2), np.zeros_like(ux)], axis=1)
    F = rng.standard_normal((3, 2, N // 2 + 1)) + 1j * rng.standard_normal((3, 2, N // 2 + 1))
    X = O.phat(F)
    Y = O.srp_scores(O.steering(O.tdoa_farfield(mic, dirs, fs, c), N), X)
    r = np.fft.irfft(X, n=N, axis=1)
    for t in range(3):
        for a, n in enumerate(lags):
            g = (N * r[t, n % N] + X[t, 0].real + X[t, N // 2].real * (-1.0) ** int(n)) / 2
            assert Y[t, a] == pytest.approx(g, abs=1e-9)


@pytest.mark.parametrize("arr,lvl", [("linear", 2), ("planar", 2), ("3d", 2)])
def test_noiseless_plane_wave_localises_to_grid_point_eq2_to_eq6(arr, lvl):
    mic = {"linear": I.array_linear_1d(), "planar": I.array_planar_2d_circle(), "3d": I.array_3d()}[arr]
    dirs = I.icosphere(lvl)
    fs, c, N = 16000.0, 343.0, 128
    tau = O.tdoa_farfield(mic, dirs, fs, c)
    W = O.steering(tau, N)
    cls = O.direction_classes(tau)
    L = W.shape[1]
    for q0 in [0, 17, 101, 161]:
        X = O.phat(_noiseless_frames(mic, dirs[q0], 2, N, fs, c))
        Y = O.srp_scores(W, X)
        idx, best = O.argmax_lowest(Y)
        assert np.all(cls[idx] == cls[q0])
        assert Y[0, q0] == pytest.approx(L, rel=1e-9)
        assert np.all(best <= L * (1 + 1e-12))


def test_noiseless_spherical_wave_localises_to_its_position_eq1():
    """A noiseless point source at candidate position q0 delays microphone m by
    fs/c ||s - r_m|| samples; with the Eq. 1 table its PHAT cross spectra are conj(W_q0), so
    Y_q0 = L and q0's class is the SRP-PHAT argmax (this fixes the generator's sign against
    Eq. 1 and Eq. 4).  The same direction at another radius is a different point."""
    mic = I.array_3d()
    pts = I.nearfield_points(1, radii=(0.3, 0.6, 1.2))          # 126 positions
    fs, c, N = 16000.0, 343.0, 128
    tau = O.tdoa_nearfield(mic, pts, fs, c)
    W = O.steering(tau, N)
    cls = O.direction_classes(tau)
    L = W.shape[1]
    for q0 in [0, 40, 77, 125]:
        src = np.repeat(pts[q0][None, :], 2, axis=0)
        fr = I.spherical_wave_frames(np.random.default_rng(q0), mic, N, fs, c, src, np.full(2, 400.0),
                                     dtype=np.complex128)
        Y = O.srp_scores(W, O.phat(fr))
        idx, best = O.argmax_lowest(Y)
        assert np.all(idx == q0) and np.all(cls[idx] == q0)
        assert Y[0, q0] == pytest.approx(L, rel=1e-9)
        assert np.all(best <= L * (1 + 1e-12))


# ---------------------------------------------------------------------------- eigen / SVD

def test_jacobi_2x2_closed_form():
    lam, U = O.jacobi_eigh(np.array([[2.0, 1 + 1j], [1 - 1j, 3.0]]))
    assert lam == pytest.approx([4.0, 1.0], abs=1e-14)
    G = np.array([[2.0, 1 + 1j], [1 - 1j, 3.0]])
    assert np.allclose(G @ U, U * lam[None, :], atol=1e-14)


def test_jacobi_matches_lapack_and_reconstructs():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((40, 40)) + 1j * rng.standard_normal((40, 40))
    G = A @ A.conj().T
    lam, U = O.jacobi_eigh(G)
    lam2 = np.linalg.eigvalsh(G)[::-1]
    assert np.max(np.abs(lam - lam2)) < 1e-11 * np.abs(lam2).max()
    assert np.max(np.abs(U.conj().T @ U - np.eye(40))) < 1e-12
    assert np.max(np.abs((U * lam) @ U.conj().T - G)) < 1e-11 * np.abs(G).max()


@pytest.mark.slow
def test_jacobi_matches_lapack_on_the_q642_line_array_gram():
    """The 1-D 7-mic line array on the level-3 grid (Q = 642, N = 512, L = 5397): the basis the
    GPU parity tests take from the oracle's own Jacobi iteration (n = Q = 642) has LAPACK's
    singular values, rank (Eq. 11) and subspace."""
    tau = O.tdoa_farfield(I.array_linear_1d(), I.icosphere(3), 16000.0, 343.0)
    W = O.steering(tau, 512)
    bj = O.svd_basis(W, 1e-5)
    assert bj["eig"] == "jacobi"
    bl = O.svd_basis(W, 1e-5, eig="lapack")
    assert bj["K"] == bl["K"]
    assert np.max(np.abs(bj["sigma2"] - bl["sigma2"])) < 1e-11 * bl["sigma2"][0]
    assert np.sum(bj["sigma2"]) == pytest.approx(W.shape[0] * W.shape[1], rel=1e-12)   # Tr = Q L
    G = bj["V"].conj().T @ bl["V"]                                                   # same subspace
    assert np.max(np.abs(G.conj().T @ G - np.eye(bj["K"]))) < 1e-10


def _small_W(arr="3d", lvl=2, N=32):
    mic = {"linear": I.array_linear_1d(), "planar": I.array_planar_2d_table(), "3d": I.array_3d()}[arr]
    tau = O.tdoa_farfield(mic, I.icosphere(lvl), 16000.0, 343.0)
    return tau, O.steering(tau, N)


@pytest.mark.parametrize("arr,lvl,N", [("3d", 2, 32), ("planar", 1, 128), ("linear", 2, 16)])
def test_svd_basis_invariants_eq10_to_eq13(arr, lvl, N):
    tau, W = _small_W(arr, lvl, N)
    Q, L = W.shape
    delta = 1e-5
    b = O.svd_basis(W, delta, eig="jacobi")
    K, V, D = b["K"], b["V"], b["D"]
    assert b["trace"] == pytest.approx(Q * L, rel=1e-14)
    assert np.sum(b["sigma2"]) == pytest.approx(Q * L, rel=1e-12)       # sum sigma^2 = Tr
    assert np.max(np.abs(V.conj().T @ V - np.eye(K))) < 1e-10              # orthonormal V
    assert np.allclose(D, W @ V)                                            # D = W V = U S
    Dn2 = np.sum(np.abs(D) ** 2, axis=1)
    assert np.mean(1 - Dn2 / L) <= delta * (1 + 1e-9)                       # Eq. 11 trace rule
    assert np.sum(b["sigma2"][:K]) >= (1 - delta) * Q * L                   # Eq. 11
    K0 = O.rank_from_delta(b["sigma2"], b["trace"], delta, close_clusters=False)
    assert K0 == 1 or np.sum(b["sigma2"][:K0 - 1]) < (1 - delta) * Q * L   # ... and smallest
    assert K >= K0 and (K == K0 or b["sigma2"][K0 - 1] - b["sigma2"][K - 1] < 1e-9 * b["sigma2"][0])
    assert K == len(b["sigma2"]) or b["sigma2"][K - 1] - b["sigma2"][K] > 1e-9 * b["sigma2"][0]
    # agrees with LAPACK's decomposition
    b2 = O.svd_basis(W, delta, eig="lapack")
    assert b2["K"] == K
    P1, P2 = V @ V.conj().T, b2["V"] @ b2["V"].conj().T                   # same subspace
    assert np.max(np.abs(P1 - P2)) < 1e-8


def test_svd_matches_numpy_svd_singular_values():
    tau, W = _small_W("3d", 1, 32)
    s = np.linalg.svd(W, compute_uv=False)
    b = O.svd_basis(W, 1e-5, eig="jacobi")
    n = len(s)
    assert np.allclose(b["sigma2"][:n], s ** 2, rtol=0, atol=1e-12 * s[0] ** 2)


def test_full_rank_svd_phat_equals_srp_phat_eq9_eq14():
    """At K = rank(W), Re{D Z} = Re{U S V^H X} = Re{W X} for any X."""
    rng = np.random.default_rng(7)
    mic = I.array_random_ball(rng, 3)
    tau = O.tdoa_farfield(mic, I.icosphere(1), 16000.0, 343.0)  # Q = 42
    W = O.steering(tau, 16)  # L = 3 * 9 = 27 < Q
    b = O.svd_basis(W, 1e-5, eig="jacobi", K=27)
    F = rng.standard_normal((6, 3, 9)) + 1j * rng.standard_normal((6, 3, 9))
    X = O.phat(F)
    Ysvd = O.svd_scores(b["D"], O.project(b["V"], X))
    Ysrp = O.srp_scores(W, X)
    assert np.max(np.abs(Ysvd - Ysrp)) < 1e-9 * W.shape[1]
    # and the Q <= L branch of the oracle, on another case
    tau2, W2 = _small_W("3d", 0, 32)   # Q = 12 < L = 357
    b2 = O.svd_basis(W2, 0.0, eig="jacobi", K=12)
    X2 = O.phat(rng.standard_normal((4, 7, 17)) + 1j * rng.standard_normal((4, 7, 17)))
    assert np.max(np.abs(O.svd_scores(b2["D"], O.project(b2["V"], X2)) - O.srp_scores(W2, X2))) < 1e-9 * 357


def test_truncated_svd_phat_close_to_srp():
    tau, W = _small_W("3d", 2, 32)
    b = O.svd_basis(W, 1e-5)
    rng = np.random.default_rng(8)
    X = O.phat(rng.standard_normal((20, 7, 17)) + 1j * rng.standard_normal((20, 7, 17)))
    Ysvd = O.svd_scores(b["D"], O.project(b["V"], X))
    Ysrp = O.srp_scores(W, X)
    # ||W - W_K||_2 <= sqrt(delta Q L) bounds every score error for ||X|| = sqrt(L)
    bound = math.sqrt(1e-5 * W.shape[0] * W.shape[1]) * math.sqrt(W.shape[1])
    assert np.max(np.abs(Ysvd - Ysrp)) <= bound
    assert np.max(np.abs(Ysvd - Ysrp)) > 0


def test_paper_gains_table1_table2():
    """Table 1 parameters with the Table 2 arrays and delta = 1e-5 give K with Q/K = 320,
    53, 36 (Section 4) -- the paper's only performance figures."""
    g = GOLD["gain_q_over_k_at_delta_1e-5"]
    t1 = GOLD["table1_parameters"]
    pos = GOLD["table2_positions_cm"]
    dirs = I.icosphere(I.icosphere_level_for(t1["Q"]))
    for arr in ("1d", "2d", "3d"):
        mic = np.array(pos[arr], dtype=np.float64) / 100.0
        W = O.steering(O.tdoa_farfield(mic, dirs, t1["fs"], t1["c"]), t1["N"])
        lam = np.linalg.eigvalsh(W @ W.conj().T)[::-1]
        K = O.rank_from_delta(np.clip(lam, 0, None), float(np.sum(np.abs(W) ** 2)), g["delta"])
        assert int(t1["Q"] / K) == g[arr], (arr, K)
        assert K == O.rank_from_delta(np.clip(lam, 0, None), float(np.sum(np.abs(W) ** 2)), g["delta"],
                                      close_clusters=False)


def test_table2_arrays_match_inputs_module():
    pos = GOLD["table2_positions_cm"]
    assert np.allclose(np.array(pos["1d"]) / 100, I.array_linear_1d())
    assert np.allclose(np.array(pos["2d"]) / 100, I.array_planar_2d_table())
    assert np.allclose(np.array(pos["3d"]) / 100, I.array_3d())


# ---------------------------------------------------------------------------- NN (Eq. 15)

def test_nn_identity_eq15_and_brute_force():
    tau, W = _small_W("3d", 2, 32)
    b = O.svd_basis(W, 1e-5)
    rng = np.random.default_rng(9)
    X = O.phat(rng.standard_normal((30, 7, 17)) + 1j * rng.standard_normal((30, 7, 17)))
    Z = O.project(b["V"], X)
    Zh = Z / np.linalg.norm(Z, axis=1, keepdims=True)
    lhs = (Zh @ b["Dhat"].T).real
    rhs = 1 - 0.5 * np.sum(np.abs(b["Dhat"][None, :, :] - np.conj(Zh)[:, None, :]) ** 2, axis=2)
    assert np.max(np.abs(lhs - rhs)) < 1e-12
    idx, d2 = O.nn_brute(b["Dhat"], Z)
    assert np.array_equal(idx, np.argmax(lhs, axis=1))
    # exhaustive and NN forms agree where ||D_q|| is nearly constant (Section 3)
    ex, _ = O.argmax_lowest(O.svd_scores(b["D"], Z))
    assert np.mean(ex == idx) > 0.9


def test_score_row_matches_srp_row():
    tau, W = _small_W("planar", 1, 64)
    rng = np.random.default_rng(10)
    X = O.phat(rng.standard_normal((5, 7, 33)) + 1j * rng.standard_normal((5, 7, 33)))
    q = np.array([0, 3, 9, 20, 41])
    assert np.allclose(O.score_row(tau, q, X, 64), O.srp_scores(W, X)[np.arange(5), q], atol=1e-10)


# ---------------------------------------------------------------------------- classes

def test_direction_classes_symmetry():
    """Planar array: mirror images across its plane share a TDOA vector; 3-D array: none."""
    dirs = I.icosphere(2)
    tau = O.tdoa_farfield(I.array_planar_2d_circle(), dirs, 16000, 343)
    cls = O.direction_classes(tau)
    for q in range(len(dirs)):
        m = np.nonzero(np.all(np.abs(dirs - dirs[q] * np.array([1, 1, -1])) < 1e-12, axis=1))[0]
        assert len(m) == 1 and cls[m[0]] == cls[q]
    tau3 = O.tdoa_farfield(I.array_3d(), dirs, 16000, 343)
    assert len(np.unique(O.direction_classes(tau3))) == len(dirs)


# ---------------------------------------------------------------------------- planted mistakes

def test_pins_catch_planted_mistakes(monkeypatch):
    """Plant plausible mistakes in (a copy of) the oracle and check a pin fails."""
    mic, dirs, fs, c, N = I.array_3d(), I.icosphere(2), 16000.0, 343.0, 128
    tau = O.tdoa_farfield(mic, dirs, fs, c)
    X = O.phat(_noiseless_frames(mic, dirs[17], 1, N, fs, c))
    # (a) wrong TDOA sign -> the plane-wave pin no longer localises to q0
    Wbad = O.steering(-tau, N)
    assert O.argmax_lowest(O.srp_scores(Wbad, X))[0][0] != 17
    # (b) conjugated steering (Eq. 4 sign) -> same
    assert O.argmax_lowest(O.srp_scores(np.conj(O.steering(tau, N)), X))[0][0] != 17
    # (c) conjugated Eq. 14 reading breaks the full-rank identity
    rng = np.random.default_rng(11)
    mic2 = I.array_random_ball(rng, 3)
    W2 = O.steering(O.tdoa_farfield(mic2, I.icosphere(1), fs, c), 16)
    b = O.svd_basis(W2, 1e-5, eig="jacobi", K=27)
    X2 = O.phat(rng.standard_normal((3, 3, 9)) + 1j * rng.standard_normal((3, 3, 9)))
    Z2 = O.project(b["V"], X2)
    bad = (np.conj(Z2) @ b["D"].T).real
    assert np.max(np.abs(bad - O.srp_scores(W2, X2))) > 1e-3
    # (d) dropping the Nyquist bin changes the row norm pin
    assert not np.allclose(np.sum(np.abs(O.steering(tau, N)[:, :-1]) ** 2, axis=1), W2.shape[1])
