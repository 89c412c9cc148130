"""Pins of the learned-proposal oracle (oracle/learned.py) against things fixed outside it:
central finite differences of the loss, closed forms at zero weights, the first Adam step,
library bfloat16 rounding, the nesting of icosphere grids, and the reduction of the search
to Eq. 14's exhaustive argmax."""
import numpy as np
import pytest
import torch

import oracle as O
import oracle.learned as OL
from paper_1811_11785_gb300 import inputs as I


def _net(rng, F=6, H1=5, H2=7, C=4, scale=0.7):
    return dict(W1=rng.normal(0, scale, (H1, F)), b1=rng.normal(0, 0.1, H1), W2=rng.normal(0, scale, (H2, H1)),
                b2=rng.normal(0, 0.1, H2), W3=rng.normal(0, scale, (C, H2)), b3=rng.normal(0, 0.1, C))


def test_gradients_match_central_differences():
    rng = np.random.default_rng(1)
    p = _net(rng)
    x = rng.normal(size=(9, 6))
    y = rng.integers(0, 4, size=9)
    _, g = OL.loss_and_grads(p, x, y)
    h = 1e-6
    for name in OL.PARAM_NAMES:
        it = np.nditer(p[name], flags=["multi_index"])
        for _ in it:
            i = it.multi_index
            q = {k: v.copy() for k, v in p.items()}
            q[name][i] += h
            lp, _ = OL.loss_and_grads(q, x, y)
            q[name][i] -= 2 * h
            lm, _ = OL.loss_and_grads(q, x, y)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[name][i]) <= 1e-7 * max(1.0, abs(fd)), (name, i, fd, g[name][i])


def test_zero_network_closed_form():
    """All weights and biases 0: every logit is 0, the loss is log C and the output-bias
    gradient is the mean of (1/C - onehot)."""
    C = 5
    p = dict(W1=np.zeros((3, 4)), b1=np.zeros(3), W2=np.zeros((3, 3)), b2=np.zeros(3), W3=np.zeros((C, 3)),
             b3=np.zeros(C))
    x = np.random.default_rng(2).normal(size=(6, 4))
    y = np.array([0, 1, 1, 4, 2, 0])
    loss, g = OL.loss_and_grads(p, x, y)
    assert abs(loss - np.log(C)) < 1e-15
    expect = np.full(C, 1.0 / C) - np.bincount(y, minlength=C) / len(y)
    assert np.allclose(g["b3"], expect, atol=1e-15)
    for name in ["W1", "b1", "W2", "b2", "W3"]:      # relu(0) = 0 blocks everything below
        assert np.all(g[name] == 0)


def test_first_adam_step_closed_form():
    """After one step from m = v = 0 the bias-corrected update is lr g / (|g| + eps)."""
    rng = np.random.default_rng(3)
    p = _net(rng)
    g = {k: rng.normal(size=v.shape) for k, v in p.items()}
    p0 = {k: v.copy() for k, v in p.items()}
    st = {}
    OL.adam_step(p, g, st, lr=1e-3)
    for k in p:
        assert np.allclose(p0[k] - p[k], 1e-3 * g[k] / (np.abs(g[k]) + 1e-8), rtol=1e-12, atol=0)


def test_softmax_and_top_cells():
    lg = np.array([[1.0, 3.0, 3.0, -2.0, 0.5], [0.0, 0.0, 0.0, 0.0, 0.0]])
    p = OL.softmax(lg)
    assert np.allclose(p.sum(axis=1), 1.0)
    assert np.array_equal(OL.top_cells(lg, 3), [[1, 2, 0], [0, 1, 2]])


def test_round_bf16_matches_torch():
    x = np.random.default_rng(4).normal(size=4096) * np.exp(np.random.default_rng(5).normal(size=4096) * 4)
    x = np.concatenate([x, [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.0e38, 1e-40]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(OL.round_bf16(x), ref)


def test_children_partition_and_nesting():
    """Levels of the icosphere are nested (the coarse vertices are the first fine ones), so
    fine direction c < C is in cell c; every fine direction is in exactly one cell."""
    coarse, fine = I.icosphere(2), I.icosphere(4)
    cell = OL.child_cells(fine, coarse)
    C = coarse.shape[0]
    assert np.array_equal(cell[:C], np.arange(C))
    kids = OL.children(cell, C)
    assert sum(len(k) for k in kids) == fine.shape[0]
    assert np.array_equal(np.sort(np.concatenate(kids)), np.arange(fine.shape[0]))
    assert min(len(k) for k in kids) >= 1
    # the nearest cell by dot product is the nearest by angle (angles within 1e-6 rad tie)
    ang = np.arccos(np.clip(fine @ coarse.T, -1, 1))
    near = ang <= ang.min(axis=1, keepdims=True) + 1e-6
    assert np.array_equal(cell, np.argmax(near, axis=1))
    assert np.sum(near.sum(axis=1) > 1) > 0        # the grids do have exact halfway points


def test_features_unit_norm_and_zero():
    Z = np.array([[3 + 4j, 0], [0, 0]], dtype=np.complex128)
    x = OL.features(Z)
    assert np.allclose(x[0], [0.6, 0.8, 0, 0]) and np.all(x[1] == 0)


def _small_problem(seed=6, T=40):
    rng = np.random.default_rng(seed)
    mic = I.array_3d()
    dirs = I.icosphere(3)
    tau = O.tdoa_farfield(mic, dirs, 16000.0, 343.0)
    W = O.steering(tau, 64)
    ob = O.svd_basis(W, 1e-5)
    src = I.random_directions(rng, T)[:, None, :]
    fr = I.plane_wave_frames(rng, mic, T, 64, 16000.0, 343.0, src, np.full(T, 10.0))
    Z = O.project(ob["V"], O.phat(fr))
    return dirs, ob, Z


def test_search_reduces_to_exhaustive():
    """theta above 1 (every frame falls back) or all cells proposed: Eq. 14's argmax."""
    dirs, ob, Z = _small_problem()
    cells = I.icosphere(1)
    kids = OL.children(OL.child_cells(dirs, cells), cells.shape[0])
    rng = np.random.default_rng(7)
    p = {k: v for k, v in _net(rng, F=2 * ob["K"], H1=8, H2=8, C=cells.shape[0]).items()}
    lg = OL.forward(p, OL.features(Z))["logits"]
    ref, _ = O.argmax_lowest(O.svd_scores(ob["D"], Z))
    i1, _, fb = OL.learned_search(ob["D"], Z, lg, kids, 4, theta=1.5)
    assert fb.all() and np.array_equal(i1, ref)
    i2, s2, fb2 = OL.learned_search(ob["D"], Z, lg, kids, cells.shape[0], theta=0.0)
    assert not fb2.any() and np.array_equal(i2, ref)
    assert np.allclose(s2, O.svd_scores(ob["D"], Z)[np.arange(len(ref)), ref])


def test_search_with_the_true_cell_on_top():
    """Logits that put the cell of the exhaustive argmax first (one-hot, confident) give the
    exhaustive answer from that cell's children alone."""
    dirs, ob, Z = _small_problem(seed=8)
    cells = I.icosphere(1)
    cell_of = OL.child_cells(dirs, cells)
    kids = OL.children(cell_of, cells.shape[0])
    ref, _ = O.argmax_lowest(O.svd_scores(ob["D"], Z))
    lg = np.full((Z.shape[0], cells.shape[0]), -30.0)
    lg[np.arange(Z.shape[0]), cell_of[ref]] = 30.0
    idx, _, fb = OL.learned_search(ob["D"], Z, lg, kids, 1, theta=0.9)
    assert not fb.any() and np.array_equal(idx, ref)
