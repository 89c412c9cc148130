"""Near-field steering (Eq. 1): the CUDA path through the C ABI against the FP64 oracle.

The offline TDOA table is the only step that changes (Section 2 derives Eq. 2 from Eq. 1 for
a distant source); everything after it runs the same kernels, so these tests pin the table
bit-exactly, the per-microphone delays of online step 4 (d_m = -fs/c ||s_q - r_m||) through
the step-4 score, and the searches on spherical-wave frames.  Tolerances as in the far-field
parity tests.
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1811_11785_gb300 as sp
from paper_1811_11785_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FS, C, N = 16000.0, 343.0, 512
_CACHE = {}


def _setup():
    if "d" in _CACHE:
        return _CACHE["d"]
    import __graft_entry__
    __graft_entry__.build()
    rng = np.random.default_rng([I.SEED_BASE + 9, 1])
    mic = I.array_3d()
    pts = I.nearfield_points(2, radii=(0.3, 0.6, 1.2))           # 486 candidate positions
    T = 400
    truth = rng.integers(0, pts.shape[0], size=T)
    frames = I.spherical_wave_frames(rng, mic, N, FS, C, pts[truth], rng.uniform(0.0, 20.0, size=T))
    tau = O.tdoa_nearfield(mic, pts, FS, C)
    W = O.steering(tau, N)
    ob = O.svd_basis(W, 1e-5)
    X = O.phat(frames)
    Z = O.project(ob["V"], X)
    d = dict(mic=mic, pts=pts, truth=truth, tau=tau, W=W, ob=ob, X=X, Z=Z, L=W.shape[1],
             Ysvd=O.svd_scores(ob["D"], Z), Ysrp=O.srp_scores(W, X), cls=O.direction_classes(tau))
    d["st"] = sp.build_steering_nearfield(mic, pts, FS, C, N, materialize_w=True)
    d["b"] = sp.svd_reduce(d["st"], 1e-5)
    d["frames"] = torch.from_numpy(frames).cuda()
    _CACHE["d"] = d
    return d


def _agree(d, idx, Y, margin_tol=1e-4, min_agree=0.995):
    cls = d["cls"]
    ref, _ = O.argmax_lowest(Y)
    m = O.top2_margin(Y, cls)
    same = cls[idx] == cls[ref]
    assert np.all(same[m > margin_tol]), f"{np.sum(~same[m > margin_tol])} clear frames disagree"
    assert np.mean(same) >= min_agree, np.mean(same)


def test_nearfield_tau_bit_exact():
    d = _setup()
    assert d["st"].nearfield and d["b"].steering.nearfield
    assert np.array_equal(d["st"].tau(), d["tau"])
    # a random geometry and random positions, as well
    rng = np.random.default_rng(5)
    mic = I.array_random_ball(rng, 9)
    pts = rng.normal(size=(300, 3)) * 0.8
    st = sp.build_steering_nearfield(mic, pts, 48000.0, 340.0, 256)
    assert np.array_equal(st.tau(), O.tdoa_nearfield(mic, pts, 48000.0, 340.0))


def test_nearfield_steering_w():
    d = _setup()
    Wg = d["st"].w().cpu().numpy()
    assert np.max(np.abs(Wg - d["W"])) <= 2e-6


def test_nearfield_localize_srp_and_svd():
    d = _setup()
    T = len(d["truth"])
    idx, best = sp.localize_srp(d["st"], d["frames"])
    _agree(d, idx.cpu().numpy(), d["Ysrp"])
    for prec, tol in [("fp32", 1e-5), ("fp16", 2e-3)]:
        idx, score, proj = sp.localize(d["b"], d["frames"], "svd_exhaustive", prec)
        torch.cuda.synchronize()
        sp.check_status()
        idx = idx.cpu().numpy()
        _agree(d, idx, d["Ysvd"])
        assert np.max(np.abs(proj.cpu().numpy() - d["Ysvd"][np.arange(T), idx])) <= tol * d["L"]
        sref = O.score_row(d["tau"], idx, d["X"], N)            # online step 4 with Eq. 1 delays
        assert np.max(np.abs(score.cpu().numpy() - sref)) <= 1e-5 * d["L"]
    # the frames come from grid points at 0-20 dB: the search finds most of them exactly
    assert np.mean(d["cls"][idx] == d["cls"][d["truth"]]) >= 0.9


def test_nearfield_basis_roundtrip(tmp_path):
    d = _setup()
    path = str(tmp_path / "near.svdphat")
    d["b"].save(path)
    b2 = sp.load_basis(path)
    assert b2.steering.nearfield
    assert np.array_equal(b2.steering.tau(), d["tau"])
    r1 = sp.localize(d["b"], d["frames"], "svd_exhaustive", "fp16")
    r2 = sp.localize(b2, d["frames"], "svd_exhaustive", "fp16")
    for a, b in zip(r1, r2):
        assert torch.equal(a, b)
    sp.check_status()
