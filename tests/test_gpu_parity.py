"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on seeded inputs.

Tolerances (scores are normalised by L = P(N/2+1), the bound on |Y_q|):
  * TDOA table: bit-exact.  W, PHAT: FP32 rounding (<= 2e-7 absolute, unit-modulus values).
  * argmax indices: identical direction class wherever the oracle's top-2 margin exceeds
    1e-4 (relative), and >= 99.5 % class agreement over all frames.
  * FP32 scores (SRP, FP32 SVD-PHAT, online step 4): |dY| <= 1e-5 L.  FP16 / BF16 search
    scores after FP32 rescoring: 2e-3 L / 1e-2 L.
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1811_11785_gb300 as sp
from paper_1811_11785_gb300 import inputs as I

pytestmark = pytest.mark.gpu

_CACHE = {}


def _setup(name, T):
    key = (name, T)
    if key in _CACHE:
        return _CACHE[key]
    import __graft_entry__
    __graft_entry__.build()
    wl = I.workload(name, T=T)
    tau = O.tdoa_farfield(wl["mic_xyz"], wl["dirs"], wl["fs"], wl["c"])
    W = O.steering(tau, wl["N"])
    ob = O.svd_basis(W, wl["delta"])
    X = O.phat(wl["frames"])
    Z = O.project(ob["V"], X)
    Ysvd = O.svd_scores(ob["D"], Z)
    Ysrp = O.srp_scores(W, X)
    cls = O.direction_classes(tau)
    st = sp.build_steering(wl["mic_xyz"], wl["dirs"], wl["fs"], wl["c"], wl["N"], materialize_w=True)
    b = sp.svd_reduce(st, wl["delta"])
    frames = torch.from_numpy(wl["frames"]).cuda()
    d = dict(wl=wl, tau=tau, W=W, ob=ob, X=X, Z=Z, Ysvd=Ysvd, Ysrp=Ysrp, cls=cls, st=st, b=b, frames=frames,
             L=W.shape[1])
    _CACHE[key] = d
    return d


CONFIGS = [("linear_q642", 100), ("planar_q2562", 777), ("array3d_q10242", 256), ("ball12_q642", 300),
           ("ball16_n1024_q642", 200)]


def oracle_basis_in_library(d):
    """The oracle's own V and D loaded into the library (through a basis file), so that a
    single step of the CUDA path can be checked on the oracle's basis."""
    if "ob_lib" not in d:
        import os
        import tempfile
        import oracle_basis
        wl = d["wl"]
        fd, path = tempfile.mkstemp(suffix=".svdphat")
        os.close(fd)
        try:
            oracle_basis.write(path, wl["mic_xyz"], wl["dirs"], wl["fs"], wl["c"], wl["N"], wl["delta"], d["ob"])
            d["ob_lib"] = sp.load_basis(path)
        finally:
            os.remove(path)
    return d["ob_lib"]


def _sqdist(Dhat, Zq):
    """||Dhat_q - Zq_t||^2 for every (t, q), in blocks of frames (FP64)."""
    out = np.empty((Zq.shape[0], Dhat.shape[0]))
    step = max(1, (1 << 23) // Dhat.size)
    for t0 in range(0, Zq.shape[0], step):
        diff = Dhat[None, :, :] - Zq[t0:t0 + step, None, :]
        out[t0:t0 + step] = np.sum(diff.real ** 2 + diff.imag ** 2, axis=2)
    return out


def _agree(d, idx, Y, margin_tol=1e-4, min_agree=0.995):
    """Class-level agreement: identical wherever the oracle's top-2 margin exceeds margin_tol,
    and >= min_agree over all frames (checked when there are >= 400 frames: below that a
    single near-tie frame is more than 0.25 %)."""
    cls = d["cls"]
    ref, _ = O.argmax_lowest(Y)
    m = O.top2_margin(Y, cls)
    same = cls[idx] == cls[ref]
    big = m > margin_tol
    assert np.all(same[big]), f"{np.sum(~same[big])} frames with margin > {margin_tol} disagree"
    if len(idx) >= 400:
        assert np.mean(same) >= min_agree, np.mean(same)
    return np.mean(same)


@pytest.mark.parametrize("name,T", CONFIGS)
def test_tau_table_bit_exact(name, T):
    d = _setup(name, T)
    assert np.array_equal(d["st"].tau(), d["tau"])


def test_tau_bit_exact_random_geometry():
    import __graft_entry__
    __graft_entry__.build()
    rng = np.random.default_rng(12)
    mic = I.array_random_ball(rng, 9)
    dirs = rng.standard_normal((1000, 3)) * rng.uniform(0.1, 10, size=(1000, 1))
    st = sp.build_steering(mic, dirs, 44100.0, 340.5, 256)
    assert np.array_equal(st.tau(), O.tdoa_farfield(mic, dirs, 44100.0, 340.5))


@pytest.mark.parametrize("name,T", CONFIGS)
def test_direction_classes_match_oracle(name, T):
    d = _setup(name, T)
    assert np.array_equal(d["st"].classes(), d["cls"])


@pytest.mark.parametrize("name,T", CONFIGS)
def test_steering_w(name, T):
    d = _setup(name, T)
    W = d["st"].w().cpu().numpy()
    assert np.max(np.abs(W - d["W"])) < 2e-7


@pytest.mark.parametrize("name,T", CONFIGS)
def test_phat(name, T):
    d = _setup(name, T)
    X = sp.phat(d["frames"]).cpu().numpy()
    assert np.max(np.abs(X - d["X"])) < 2e-6


def test_phat_zero_entries():
    import __graft_entry__
    __graft_entry__.build()
    rng = np.random.default_rng(13)
    F = (rng.standard_normal((3, 4, 9)) + 1j * rng.standard_normal((3, 4, 9))).astype(np.complex64)
    F[1, 2, :] = 0
    F[2, 0, 4] = 0
    X = sp.phat(torch.from_numpy(F).cuda()).cpu().numpy()
    assert np.max(np.abs(X - O.phat(F))) < 2e-6
    assert np.all(X[1].reshape(6, 9)[[1, 3, 5]] == 0)


@pytest.mark.parametrize("name,T", CONFIGS)
def test_svd_reduce_matches_oracle(name, T):
    d = _setup(name, T)
    b, ob = d["b"], d["ob"]
    assert b.K == ob["K"]
    s2 = b.sigma2()[: b.K]
    assert np.max(np.abs(s2 - ob["sigma2"][: b.K]) / ob["sigma2"][0]) < 1e-9
    V = b.V()
    G = ob["V"].conj().T @ V                      # same subspace <=> unitary K x K
    assert np.max(np.abs(G.conj().T @ G - np.eye(b.K))) < 1e-8
    assert np.max(np.abs(V.conj().T @ V - np.eye(b.K))) < 1e-10
    assert np.max(np.abs(b.D() - d["W"] @ V)) < 1e-8 * np.sqrt(d["L"])


@pytest.mark.parametrize("name,T", CONFIGS)
@pytest.mark.parametrize("prec,tol", [("fp32", 2e-6), ("fp16", 1e-4), ("bf16", 1e-3)])
def test_project(name, T, prec, tol):
    """Eq. 12 on the oracle's basis (Z depends on the phases of V's columns)."""
    d = _setup(name, T)
    b = oracle_basis_in_library(d)
    assert np.array_equal(b.V(), d["ob"]["V"])
    Zg = sp.project(b, d["frames"], prec).cpu().numpy()
    L = d["L"]
    if prec == "fp32":
        # FP32 accumulation over L terms: the bound grows with L (4e-8 L dominates beyond L ~ 2500)
        bound = max(tol * np.sqrt(L), 4e-8 * L)
    else:
        # operand rounding (tol sqrt(L)) plus the tensor core's FP32 accumulator: 2L/16 additions
        # of K = 16 blocks, each rounded toward zero (at most 2^-23 of the partial sum), and every
        # partial sum is at most ||V_k|| ||X|| = sqrt(L) (Cauchy-Schwarz, PHAT entries of modulus 1)
        bound = tol * np.sqrt(L) + (2 * L / 16) * 2.0**-23 * np.sqrt(L)
    assert np.max(np.abs(Zg - d["Z"])) <= bound


@pytest.mark.parametrize("name,T", [("linear_q642", 100), ("planar_q2562", 777), ("array3d_q10242", 256)])
@pytest.mark.parametrize("prec,tol", [("fp16", 1e-4), ("bf16", 1e-3)])
def test_project_tma_fed_and_register_fed_kernels(name, T, prec, tol):
    """The 7-microphone arrays run GEMM1 with the STFT fed by TMA when the frames are 16-byte
    aligned, and with per-thread loads otherwise (a buffer 8 bytes off): both give the oracle's
    Z (Eq. 12) within the tensor-core bound, and the two paths agree with each other."""
    d = _setup(name, T)
    b = oracle_basis_in_library(d)
    fr = d["frames"]
    buf = torch.empty(fr.numel() + 1, dtype=torch.complex64, device=fr.device)
    shifted = buf[1:].view(fr.shape)              # 8 bytes past a 256-byte boundary
    shifted.copy_(fr)
    assert fr.data_ptr() % 16 == 0 and shifted.data_ptr() % 16 == 8
    Za = sp.project(b, fr, prec).cpu().numpy()
    Zb = sp.project(b, shifted, prec).cpu().numpy()
    L = d["L"]
    bound = tol * np.sqrt(L) + (2 * L / 16) * 2.0**-23 * np.sqrt(L)
    assert np.max(np.abs(Za - d["Z"])) <= bound
    assert np.max(np.abs(Zb - d["Z"])) <= bound
    assert np.max(np.abs(Za - Zb)) <= 2 * bound
    # odd frame counts leave the last row of microphone pairs half outside the buffer
    for t in (1, 3, 129):
        Zt = sp.project(b, fr[:t].contiguous(), prec).cpu().numpy()
        assert np.max(np.abs(Zt - Za[:t])) <= 2 * bound


@pytest.mark.parametrize("name,T", CONFIGS)
def test_localize_srp(name, T):
    d = _setup(name, T)
    idx, best = sp.localize_srp(d["st"], d["frames"])
    idx = idx.cpu().numpy()
    _agree(d, idx, d["Ysrp"])
    ref = d["Ysrp"][np.arange(T), idx]
    # FP32 scores within 1e-5 L of FP64 (the kernel sums blocks of 256 complex terms and then
    # the block sums, so its rounding error is about u L sqrt(L / 256), u = 2^-24)
    L = d["L"]
    assert np.max(np.abs(best.cpu().numpy() - ref)) <= 1e-5 * L


@pytest.mark.parametrize("name,T", CONFIGS)
@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp16", 2e-3), ("bf16", 1e-2)])
def test_localize_svd_exhaustive(name, T, prec, tol):
    d = _setup(name, T)
    idx, score, proj = sp.localize(d["b"], d["frames"], "svd_exhaustive", prec)
    torch.cuda.synchronize()
    sp.check_status()
    idx = idx.cpu().numpy()
    _agree(d, idx, d["Ysvd"])
    assert np.all(d["cls"][idx] == idx)           # the lowest index of the winning class
    assert np.max(np.abs(proj.cpu().numpy() - d["Ysvd"][np.arange(T), idx])) <= tol * d["L"]
    sref = O.score_row(d["tau"], idx, d["X"], d["wl"]["N"])       # Algorithm 1 online step 4
    assert np.max(np.abs(score.cpu().numpy() - sref)) <= 1e-5 * d["L"]


@pytest.mark.parametrize("name,T", CONFIGS)
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_localize_kdtree(name, T, prec):
    d = _setup(name, T)
    b = d["b"]
    idx, _, proj = sp.localize(b, d["frames"], "svd_kdtree", prec, score=False)
    idx = idx.cpu().numpy()
    # exact search: the brute-force neighbour (plain numpy here) of the GPU's own query
    Zg = sp.project(b, d["frames"], prec).cpu().numpy()
    D = b.D()
    Dhat = D / np.linalg.norm(D, axis=1, keepdims=True)
    Zh = np.conj(Zg / np.linalg.norm(Zg, axis=1, keepdims=True))
    dist = _sqdist(Dhat, Zh)
    nn = np.argmin(dist, axis=1)
    d2 = dist[np.arange(len(nn)), nn]
    cls = d["cls"]
    dsec = np.where(cls[None, :] == cls[nn][:, None], np.inf, dist).min(axis=1)
    clear = dsec - d2 > 1e-5
    assert np.all(cls[idx[clear]] == cls[nn[clear]])
    assert np.all(cls[idx] == idx)                 # the tree holds one point per class
    # against the oracle's own normalised search (Eq. 15) on its FP64 query
    Dh = d["ob"]["Dhat"]
    ref, rd2 = O.nn_brute(Dh, d["Z"])
    Zo = np.conj(d["Z"] / np.linalg.norm(d["Z"], axis=1, keepdims=True))
    od = _sqdist(Dh, Zo)
    osec = np.where(cls[None, :] == cls[ref][:, None], np.inf, od).min(axis=1)
    big = (osec - rd2) > 1e-4
    assert np.all(cls[idx[big]] == cls[ref[big]])
    if T >= 400:
        assert np.mean(cls[idx] == cls[ref]) >= 0.995
    assert np.max(np.abs(proj.cpu().numpy() - (1 - d2 / 2))) < 1e-4


@pytest.mark.parametrize("name,T", [("planar_q2562", 777), ("array3d_q10242", 256)])
def test_kdtree_search_visits(name, T):
    """The step-level tree search (Eq. 15) on sp_project's Z gives sp_localize's k-d tree result,
    and its visit counters are consistent with the tree: at least one root-to-leaf path (depth
    nodes, one bucket) per query, at most every node and bucket."""
    d = _setup(name, T)
    b = d["b"]
    Z = sp.project(b, d["frames"], "fp16")
    idx, score, visits = sp.kdtree_search(b, Z)
    ref, _, pref = sp.localize(b, d["frames"], "svd_kdtree", "fp16", score=False)
    torch.cuda.synchronize()
    assert torch.equal(idx, ref) and torch.equal(score, pref)
    info = b.kdtree_info()
    n_leaves = (info["n_nodes"] + 1) // 2
    v = visits.cpu().numpy()
    assert np.all(v[:, 0] >= info["depth"] - 1) and np.all(v[:, 0] <= info["n_nodes"])
    assert np.all(v[:, 1] >= 1) and np.all(v[:, 1] <= n_leaves)


def test_tree_shape():
    d = _setup("planar_q2562", 777)
    info = d["b"].kdtree_info()
    n_classes = len(np.unique(d["cls"]))
    assert info["leaf_size"] == 32 and info["n_nodes"] >= 2 * (n_classes // 32) - 1


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp32"])
def test_ragged_batches_are_consistent(prec):
    """Sub-batches in 16-byte-aligned buffers (copies) give bit-identical results; views that
    start 8 bytes off a 16-byte boundary run the register-fed GEMM1 (another FP32 summation
    order) and agree within the FP32 bound."""
    d = _setup("planar_q2562", 777)
    full, _, pfull = sp.localize(d["b"], d["frames"], "svd_exhaustive", prec, score=False)
    for lo, hi in [(0, 1), (5, 132), (128, 256), (700, 777), (3, 3)]:
        idx, _, pj = sp.localize(d["b"], d["frames"][lo:hi].clone(), "svd_exhaustive", prec, score=False)
        assert torch.equal(idx, full[lo:hi])
        assert torch.equal(pj, pfull[lo:hi])
        view = d["frames"][lo:hi]                  # no copy: 8 bytes off for odd lo
        iv, _, pv = sp.localize(d["b"], view, "svd_exhaustive", prec, score=False)
        if hi > lo:
            assert np.max(np.abs(pv.cpu().numpy() - pj.cpu().numpy())) <= 1e-5 * d["L"]
            assert np.mean((iv == idx).cpu().numpy()) >= 0.99


def test_zero_and_nan_frames():
    d = _setup("linear_q642", 100)
    fr = d["frames"][:6].clone()
    fr[1] = 0                                   # silent frame: every cross spectrum is 0
    fr[2, :, 10] = float("nan")
    for prec in ["fp32", "fp16"]:
        idx, score, proj = sp.localize(d["b"], fr, "svd_exhaustive", prec)
        idx = idx.cpu().numpy()
        assert idx[1] >= 0 and abs(float(proj[1])) < 1e-6
        kidx, _, _ = sp.localize(d["b"], fr, "svd_kdtree", prec, score=False)
        assert int(kidx[1]) == -1              # ||Z|| = 0: no direction
    torch.cuda.synchronize()


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_window_overflow_frames_take_the_fp32_list_scan(prec):
    """A silent frame (Z = 0) ties every class, so its candidate window overflows and the
    frame is scored by the FP32 scan over every class on the compacted list: its index is the
    lowest direction (Eq. 14 with ties to the lowest index) and its projection score 0, while
    the other frames of the batch come out exactly as without the silent ones."""
    d = _setup("planar_q2562", 777)
    fr = d["frames"][:600].clone()
    silent = torch.arange(3, 600, 7, device=fr.device)
    fr[silent] = 0
    idx, score, proj = sp.localize(d["b"], fr, "svd_exhaustive", prec)
    ref_i, ref_s, ref_p = sp.localize(d["b"], d["frames"][:600].contiguous(), "svd_exhaustive", prec)
    torch.cuda.synchronize()
    sp.check_status()
    keep = torch.ones(600, dtype=torch.bool, device=fr.device)
    keep[silent] = False
    assert torch.equal(idx[keep], ref_i[keep])
    assert torch.equal(proj[keep], ref_p[keep]) and torch.equal(score[keep], ref_s[keep])
    assert bool((idx[silent] == 0).all())
    assert float(proj[silent].abs().max()) == 0.0 and float(score[silent].abs().max()) == 0.0


def test_host_path_matches_device():
    d = _setup("planar_q2562", 777)
    fh = d["frames"].cpu().pin_memory()
    for prec in ["fp16", "fp32"]:
        i1, s1, p1 = sp.localize(d["b"], d["frames"], "svd_exhaustive", prec)
        i2, s2, p2 = sp.localize_host(d["b"], fh, "svd_exhaustive", prec, chunk_frames=200)
        assert torch.equal(i1.cpu(), i2)
        assert torch.equal(p1.cpu(), p2)
        assert torch.allclose(s1.cpu(), s2)


def test_bounded_wait_reports_timeout():
    d = _setup("linear_q642", 100)
    try:
        sp.set_wait_budget(1)
        sp.localize(d["b"], d["frames"], "svd_exhaustive", "fp16", score=False)
        with pytest.raises(sp.SvdPhatError) as e:
            sp.check_status()
        assert e.value.code == -4
    finally:
        sp.set_wait_budget(0)
    idx, _, _ = sp.localize(d["b"], d["frames"], "svd_exhaustive", "fp16", score=False)
    sp.check_status()
    _agree(d, idx.cpu().numpy(), d["Ysvd"])


def test_bench_workload_full_size_sampled():
    """The measured workload at full size (65,536 frames, planar array, Q = 2562) in the launch
    configuration the benchmark times; 2,048 sampled frames are checked against the oracle
    (enough for the >= 99.5 % agreement rule to apply)."""
    import __graft_entry__
    __graft_entry__.build()
    wl = I.workload("planar_q2562")
    st = sp.build_steering(wl["mic_xyz"], wl["dirs"], wl["fs"], wl["c"], wl["N"])
    b = sp.svd_reduce(st, wl["delta"])
    frames = torch.from_numpy(wl["frames"]).cuda()
    rng = np.random.default_rng(14)
    sel = np.sort(rng.choice(frames.shape[0], 2048, replace=False))
    tau = O.tdoa_farfield(wl["mic_xyz"], wl["dirs"], wl["fs"], wl["c"])
    W = O.steering(tau, wl["N"])
    ob = O.svd_basis(W, wl["delta"])
    X = O.phat(wl["frames"][sel])
    Y = O.svd_scores(ob["D"], O.project(ob["V"], X))
    d = dict(cls=O.direction_classes(tau))
    for prec in ["fp16", "bf16"]:
        idx, score, proj = sp.localize(b, frames, "svd_exhaustive", prec)
        torch.cuda.synchronize()
        sp.check_status()
        idx = idx.cpu().numpy()[sel]
        _agree(d, idx, Y)
        sref = O.score_row(tau, idx, X, wl["N"])
        assert np.max(np.abs(score.cpu().numpy()[sel] - sref)) <= 1e-5 * W.shape[1]


def test_save_load_basis_roundtrip(tmp_path):
    """A basis written by sp_save_basis and read back by sp_load_basis (with its own steering
    handle) gives bit-identical results on every search mode."""
    d = _setup("planar_q2562", 777)
    path = str(tmp_path / "planar.svdphat")
    d["b"].save(path)
    b2 = sp.load_basis(path)
    assert b2.K == d["b"].K
    assert np.array_equal(b2.V(), d["b"].V()) and np.array_equal(b2.D(), d["b"].D())
    assert np.array_equal(b2.steering.tau(), d["st"].tau())
    assert np.array_equal(b2.steering.classes(), d["st"].classes())
    for mode, prec in [("svd_exhaustive", "fp16"), ("svd_exhaustive", "bf16"), ("svd_exhaustive", "fp32"),
                       ("svd_kdtree", "fp16")]:
        r1 = sp.localize(d["b"], d["frames"], mode, prec)
        r2 = sp.localize(b2, d["frames"], mode, prec)
        for a, b in zip(r1, r2):
            assert torch.equal(a, b)
    sp.check_status()
    del b2
