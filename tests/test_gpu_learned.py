"""Parity of the learned proposal's CUDA path (through the C ABI) with the FP64 oracle of
oracle/learned.py, on the 3-D 7-mic array with the level-5 grid (Q = 10242, K = 71) and the
642 cells of the level-3 grid.

Steps are checked on the oracle's own basis, loaded into the library from a basis file:
  * cells: bit-exact;
  * FP32 forward / gradient / Adam against the FP64 forward, chain-rule gradient and Adam on
    the same parameters and rows (relative 1e-4 of the largest entry);
  * tensor-core inference (BF16 weights and activations) against the FP64 forward on the
    BF16-rounded weights and activations (|d logit| <= 5e-3 (1 + |logit|)), top-8 cells
    where the oracle's order is clear;
  * the search against the oracle's search where its cell choice and its winner are clear;
  * training: the trained network finds the exhaustive answer's cell and cuts the scan.
"""
import numpy as np
import pytest
import torch

import oracle as O
import oracle.learned as OL
import paper_1811_11785_gb300 as sp
from paper_1811_11785_gb300 import inputs as I
from test_gpu_parity import _agree, _setup, oracle_basis_in_library

pytestmark = pytest.mark.gpu

NAME, T = "array3d_q10242", 256
CELL_LEVEL = 3


def _ctx():
    d = _setup(NAME, T)
    if "cells" not in d:
        d["cells"] = I.icosphere(CELL_LEVEL)
        d["cell_of"] = OL.child_cells(d["wl"]["dirs"], d["cells"])
        d["kids"] = OL.children(d["cell_of"], d["cells"].shape[0])
    return d


def _params(p, seed):
    return I.mlp_params(np.random.default_rng(seed), p.F, p.H1, p.H2, p.C)


def test_cells_bit_exact():
    d = _ctx()
    p = sp.Proposal(oracle_basis_in_library(d), d["cells"], seed=1)
    assert np.array_equal(p.cells(), d["cell_of"])
    assert p.F == 2 * d["ob"]["K"] and p.C == 642


def test_forward_and_gradient_match_oracle():
    d = _ctx()
    p = sp.Proposal(oracle_basis_in_library(d), d["cells"], seed=1)
    theta = _params(p, 11)
    p.set_params(theta)
    assert np.array_equal(p.get_params(), theta)
    rng = np.random.default_rng(12)
    x = rng.normal(size=(300, p.F))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    y = rng.integers(0, p.C, size=300)
    y[7] = -1                                        # an invalid label contributes nothing
    xt = torch.from_numpy(x.astype(np.float32)).cuda()
    yt = torch.from_numpy(y.astype(np.int32)).cuda()
    P = OL.unflatten(theta.astype(np.float64), p.F, p.H1, p.H2, p.C)
    x32 = x.astype(np.float32).astype(np.float64)
    ref = OL.forward(P, x32)["logits"]
    lg = p.forward_f32(xt).cpu().numpy()
    assert np.max(np.abs(lg - ref)) <= 1e-4 * max(1.0, np.max(np.abs(ref)))
    g, loss = p.grad(xt, yt)
    keep = y >= 0
    lo, gref = OL.loss_and_grads(P, x32[keep], y[keep])
    gref = OL.flatten(gref) * keep.sum() / len(y)    # the mean runs over all n rows
    lo = lo * keep.sum() / len(y)
    gg = g.cpu().numpy()
    assert abs(float(loss) - lo) <= 1e-5 * lo
    assert np.max(np.abs(gg - gref)) <= 1e-4 * np.max(np.abs(gref))


def test_adam_steps_match_oracle():
    d = _ctx()
    p = sp.Proposal(oracle_basis_in_library(d), d["cells"], seed=1)
    theta = _params(p, 21)
    p.set_params(theta)
    rng = np.random.default_rng(22)
    x = rng.normal(size=(300, p.F))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    x = x.astype(np.float32)
    y = rng.integers(0, p.C, size=300).astype(np.int32)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    P = OL.unflatten(theta.astype(np.float64), p.F, p.H1, p.H2, p.C)
    st = {}
    big = np.ones(p.n_params, dtype=bool)   # gradients well above FP32 noise at every step
    for step in range(2):
        rows = rng.choice(300, 128, replace=False).astype(np.int32)
        p.train_step(xt, yt, rows=torch.from_numpy(rows).cuda(), lr=1e-3)
        _, g = OL.loss_and_grads(P, x[rows].astype(np.float64), y[rows])
        g = OL.flatten(g)
        big &= np.abs(g) > 1e-4
        OL.adam_step(P, OL.unflatten(g, p.F, p.H1, p.H2, p.C), st, lr=1e-3)
        err = np.abs(p.get_params().astype(np.float64) - OL.flatten(P))
        if step == 0:
            # lr g / (|g| + eps): insensitive to the rounding of g where |g| >> eps
            assert np.max(err[big]) <= 2e-6
    # second step: mh / sqrt(vh) with mh = (0.09 g1 + 0.1 g2) / 0.19 is sensitive to FP32
    # rounding where the two gradients nearly cancel (and the second gradient is taken at
    # parameters whose first-step updates differ where |g| ~ eps): most entries still match
    # to 2e-6 and every update stays within its bound of about lr per step; a wrong moment,
    # bias correction or eps would move most entries by O(lr)
    assert np.mean(err[big] <= 2e-6) >= 0.97
    assert np.max(err) <= 4.1e-3
    assert big.mean() > 0.2


def _oracle_logits(p, theta, Z):
    P = OL.unflatten(theta.astype(np.float64), p.F, p.H1, p.H2, p.C)
    for w in ("W1", "W2", "W3"):
        P[w] = OL.round_bf16(P[w])
    return OL.forward(P, OL.features(Z), act_round=OL.round_bf16)["logits"]


def test_tensor_core_inference_matches_oracle():
    d = _ctx()
    b = oracle_basis_in_library(d)
    p = sp.Proposal(b, d["cells"], seed=1)
    theta = _params(p, 31)
    theta[-(p.H2 * p.C + p.C):] *= 8.0             # spread the logits (as a trained network does)
    p.set_params(theta)
    Z64 = d["Z"].astype(np.complex64)                # the oracle's Z, in the kernel's input type
    Zt = torch.from_numpy(Z64).cuda()
    zn2 = torch.from_numpy(np.sum(np.abs(Z64.astype(np.complex128)) ** 2, axis=1).astype(np.float32)).cuda()
    top, conf, lg = p.infer(Zt, zn2, logits=True)
    torch.cuda.synchronize()
    sp.check_status()
    ref = _oracle_logits(p, theta, Z64)
    lg = lg.cpu().numpy()
    assert np.max(np.abs(lg - ref) / (1 + np.abs(ref))) <= 5e-3
    pr = OL.softmax(ref)
    assert np.max(np.abs(conf.cpu().numpy() - pr.max(axis=1))) <= 2e-3
    # every reported cell holds (within tolerance) the oracle's logit of that rank, and the
    # cell itself is the oracle's wherever that rank is separated from its neighbours
    top = top.cpu().numpy()
    srt = -np.sort(-ref, axis=1)
    got = np.take_along_axis(ref, top, axis=1)
    assert np.all(np.abs(got - srt[:, :8]) <= 1e-2 * (1 + np.abs(srt[:, :8])))
    gap = np.diff(-srt[:, :9], axis=1)                 # gap[:, k] = srt[k] - srt[k + 1]
    left = np.concatenate([np.full((T, 1), np.inf), gap[:, :7]], axis=1)
    clear = (gap[:, :8] > 0.02) & (left > 0.02)
    assert clear.mean() > 0.3
    assert np.array_equal(top[clear], OL.top_cells(ref, 8)[clear])


@pytest.mark.parametrize("theta_mode", ["never", "always", "median"])
def test_learned_search_matches_oracle(theta_mode):
    d = _ctx()
    b = oracle_basis_in_library(d)
    p = sp.Proposal(b, d["cells"], seed=1)
    params = _params(p, 41)
    # a confident untrained network: output layer scaled so that logits spread widely
    n3 = p.H2 * p.C + p.C
    params[-n3:] *= 8.0
    p.set_params(params)
    ref_lg = _oracle_logits(p, params, d["Z"])
    conf_o = OL.softmax(ref_lg).max(axis=1)
    theta = {"never": 0.0, "always": 2.0, "median": float(np.median(conf_o))}[theta_mode]
    n_top = 4
    idx, score, proj, fb = p.localize(d["frames"], "fp16", n_top=n_top, theta=theta)
    torch.cuda.synchronize()
    sp.check_status()
    idx, proj, fb = idx.cpu().numpy(), proj.cpu().numpy(), fb.cpu().numpy()
    oi, obest, ofb = OL.learned_search(d["ob"]["D"], d["Z"], ref_lg, d["kids"], n_top, theta)
    cls, L = d["cls"], d["L"]
    decided = np.abs(conf_o - theta) > 1e-3
    assert np.array_equal(fb[decided].astype(bool), ofb[decided])
    # the cell choice is clear when the n_top-th and (n_top+1)-th logits are apart
    srt = -np.sort(-ref_lg, axis=1)
    cells_clear = srt[:, n_top - 1] - srt[:, n_top] > 0.02
    # the winner is clear when the best other class among the candidates is 1e-4 L below
    Ysvd = d["Ysvd"]
    margin = np.empty(T)
    for t in range(T):
        cand = np.arange(Ysvd.shape[1]) if ofb[t] else np.concatenate([d["kids"][c] for c in OL.top_cells(ref_lg, n_top)[t]])
        y = Ysvd[t, cand]
        other = y[cls[cand] != cls[oi[t]]]
        margin[t] = (obest[t] - (other.max() if other.size else -np.inf)) / L
    ok = decided & (cells_clear | ofb) & (margin > 1e-4)
    assert ok.mean() > 0.3
    assert np.all(cls[idx[ok]] == cls[oi[ok]])
    assert np.all(cls[idx] == idx)
    assert np.max(np.abs(proj[ok] - obest[ok])) <= 2e-3 * L
    sref = O.score_row(d["tau"], idx, d["X"], d["wl"]["N"])     # Algorithm 1 online step 4
    assert np.max(np.abs(score.cpu().numpy() - sref)) <= 1e-5 * L
    # frames that fell back ran sp_localize's exhaustive tensor-core scan on the same Z (the
    # kept-class set of the one-pass scan does not depend on the tile order; only whether a
    # frame's window overflowed on the way can, and then the FP32 list scan takes it)
    fbm = fb.astype(bool)
    if fbm.any():
        ei, _, ep = sp.localize(b, d["frames"], "svd_exhaustive", "fp16")
        ei, ep = ei.cpu().numpy()[fbm], ep.cpu().numpy()[fbm]
        same = idx[fbm] == ei
        assert same.mean() >= 0.99
        assert np.max(np.abs(proj[fbm][same] - ep[same]), initial=0.0) <= 1e-5 * L
    if theta_mode == "always":
        assert fb.all()
        _agree(d, idx, Ysvd)


EVAL_T = 2048


def _eval_set(d):
    """2,048 held-out frames of the same workload with the oracle's exhaustive answer."""
    if "eval" not in d:
        wl = I.workload(NAME, T=EVAL_T, seed_offset=1)
        X = O.phat(wl["frames"])
        Y = O.svd_scores(d["ob"]["D"], O.project(d["ob"]["V"], X))
        ref, _ = O.argmax_lowest(Y)
        d["eval"] = dict(frames=torch.from_numpy(wl["frames"]).cuda(), ref=ref, m=O.top2_margin(Y, d["cls"]))
    return d["eval"]


def test_trained_network_gain():
    """Trained on frames the method labels itself (the cell of the exhaustive argmax), the
    network's top cells hold the oracle's answer far more often than an untrained one's, and
    the learned search keeps >= 99.5 % agreement with the exhaustive oracle while most frames
    skip the exhaustive scan."""
    d = _ctx()
    wl = d["wl"]
    b = d["b"]                                     # the library's own basis (product flow)
    rng = np.random.default_rng(I.SEED_BASE + 50)
    fr, _, _ = I.training_frames(rng, wl["mic_xyz"], 65536, wl["N"], wl["fs"], wl["c"])
    frames = torch.from_numpy(fr).cuda()
    p = sp.Proposal(b, d["cells"], seed=5)
    untrained = sp.Proposal(b, d["cells"], seed=5)
    x, y = p.examples(frames, "fp16")
    losses = p.train(x, y, epochs=6, batch=512, lr=1e-3, seed=6)
    print("loss per epoch", np.round(losses, 3))
    assert losses[-1] < 0.5 * losses[0]
    ev = _eval_set(d)
    target = d["cell_of"][ev["ref"]]
    clear = ev["m"] > 1e-4
    Zg = sp.project(b, ev["frames"], "fp16")
    zn2 = (Zg.real ** 2 + Zg.imag ** 2).sum(dim=1).float()
    recall = {}
    for tag, net in (("trained", p), ("untrained", untrained)):
        top, conf, _ = net.infer(Zg, zn2)
        top = top.cpu().numpy()
        for n in (1, 4, 8):
            recall[(tag, n)] = float(np.mean(np.any(top[:, :n] == target[:, None], axis=1)[clear]))
    print("top-n recall", recall)
    assert recall[("trained", 4)] >= 0.9 and recall[("untrained", 4)] <= 0.2
    cls = d["cls"]
    table = {}
    for n_top in (4, 8):
        for theta in (0.2, 0.4, 0.6, 0.8, 0.9):
            idx, _, _, fb = p.localize(ev["frames"], "fp16", n_top=n_top, theta=theta)
            idx, fb = idx.cpu().numpy(), fb.cpu().numpy()
            table[(n_top, theta)] = (float(fb.mean()), float(np.mean(cls[idx] == cls[ev["ref"]])))
    print("(n_top, theta) -> (fallback fraction, agreement)", table)
    for key, max_fb in (((8, 0.2), 0.05), ((8, 0.4), 0.3)):
        fbf, agree = table[key]
        assert agree >= 0.995 and fbf <= max_fb, (key, fbf, agree)


def test_learned_mode_needs_a_proposal():
    d = _ctx()
    with pytest.raises(sp.SvdPhatError) as e:
        sp.localize(d["b"], d["frames"], "svd_learned", "fp16")
    assert e.value.code == -1


def test_bf16_learned_fallback_equals_exhaustive():
    """Every frame falling back (theta > 1) gives exactly the exhaustive BF16 result."""
    d = _ctx()
    p = sp.Proposal(d["b"], d["cells"], seed=3)
    li, ls, _, fb = p.localize(d["frames"], "bf16", n_top=4, theta=2.0)
    ei, es, _ = sp.localize(d["b"], d["frames"], "svd_exhaustive", "bf16")
    torch.cuda.synchronize()
    assert bool(fb.all())
    assert torch.equal(li, ei) and torch.equal(ls, es)


def test_wide_basis_inference_and_search():
    """2K = 262 features (five 64-column atoms) on the 16-mic N = 1024 array: tensor-core
    logits against the FP64 forward, and the search with every frame falling back equals the
    exhaustive result."""
    d = _setup("ball16_n1024_q642", 200)
    b = oracle_basis_in_library(d)
    cells = I.icosphere(1)
    p = sp.Proposal(b, cells, hidden=(128, 128), seed=1)
    assert p.F == 2 * d["ob"]["K"] and p.F > 256
    theta = _params(p, 51)
    theta[-(p.H2 * p.C + p.C):] *= 8.0
    p.set_params(theta)
    Z64 = d["Z"].astype(np.complex64)
    Zt = torch.from_numpy(Z64).cuda()
    zn2 = torch.from_numpy(np.sum(np.abs(Z64.astype(np.complex128)) ** 2, axis=1).astype(np.float32)).cuda()
    top, conf, lg = p.infer(Zt, zn2, logits=True)
    torch.cuda.synchronize()
    sp.check_status()
    ref = _oracle_logits(p, theta, Z64)
    assert np.max(np.abs(lg.cpu().numpy() - ref) / (1 + np.abs(ref))) <= 5e-3
    li, _, _, fb = p.localize(d["frames"], "fp16", n_top=4, theta=2.0)
    ei, _, _ = sp.localize(b, d["frames"], "svd_exhaustive", "fp16")
    torch.cuda.synchronize()
    assert bool(fb.all()) and torch.equal(li, ei)


def test_learned_search_on_a_wide_basis():
    """The 16-mic N = 1024 array (K = 131-135, 2K = 262-270: rows of 33-34 16-byte pieces, the
    screening with two rows in flight per lane group) with 42 cells of ~15 directions: with a
    confident network and no fallback, the search matches the oracle's search wherever its
    cell choice and winner are clear, and its scores are within the FP32 tolerance."""
    d = _setup("ball16_n1024_q642", 200)
    cells = I.icosphere(1)
    cell_of = OL.child_cells(d["wl"]["dirs"], cells)
    kids = OL.children(cell_of, cells.shape[0])
    b = oracle_basis_in_library(d)
    p = sp.Proposal(b, cells, seed=1)
    assert p.F == 2 * d["ob"]["K"] and p.F > 4 * 48 and np.array_equal(p.cells(), cell_of)
    params = _params(p, 51)
    params[-(p.H2 * p.C + p.C):] *= 8.0
    p.set_params(params)
    ref_lg = _oracle_logits(p, params, d["Z"])
    n_top = 4
    idx, score, proj, fb = p.localize(d["frames"], "fp16", n_top=n_top, theta=0.0)
    torch.cuda.synchronize()
    sp.check_status()
    idx, proj, fb = idx.cpu().numpy(), proj.cpu().numpy(), fb.cpu().numpy()
    assert not fb.any()
    oi, obest, ofb = OL.learned_search(d["ob"]["D"], d["Z"], ref_lg, kids, n_top, 0.0)
    cls, L, Ysvd = d["cls"], d["L"], d["Ysvd"]
    srt = -np.sort(-ref_lg, axis=1)
    cells_clear = srt[:, n_top - 1] - srt[:, n_top] > 0.02
    margin = np.empty(len(idx))
    for t in range(len(idx)):
        cand = np.concatenate([kids[c] for c in OL.top_cells(ref_lg, n_top)[t]])
        y = Ysvd[t, cand]
        other = y[cls[cand] != cls[oi[t]]]
        margin[t] = (obest[t] - (other.max() if other.size else -np.inf)) / L
    ok = cells_clear & (margin > 1e-4)
    assert ok.mean() > 0.3
    assert np.all(cls[idx[ok]] == cls[oi[ok]])
    assert np.max(np.abs(proj[ok] - obest[ok])) <= 2e-3 * L
    sref = O.score_row(d["tau"], idx, d["X"], d["wl"]["N"])
    assert np.max(np.abs(score.cpu().numpy() - sref)) <= 1e-5 * L
