"""FP64 ORACLE for the learned direction proposal -- test infrastructure, NOT the product.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` import this module; it imports
nothing from the product library.

The paper has no learned component: its searches are the exhaustive argmax of Eq. 14 and
the k-d tree of Eq. 15 (Section 3).  This module is the reference for an extra search that
narrows Eq. 14 to a few coarse cells of the direction grid, defined as follows (plain
definitions, each step written out):

* cells: the directions of a coarser grid; every direction q of the fine grid belongs to
  the cell whose direction has the largest dot product with it.  Nested grids put many
  fine directions exactly halfway between cells, so dot products within CELL_TIE (1e-12)
  of the largest count as ties and the lowest such cell index wins.  The children of a
  cell are the fine directions that belong to it.
* features of a frame: x = [Re Z_0, Im Z_0, Re Z_1, Im Z_1, ...] / ||Z|| (2K reals, Z of
  Eq. 12); x = 0 when ||Z|| = 0.
* network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), logits = W3 h2 + b3; probabilities
  by softmax; loss = mean over the batch of -log p[label] (cross-entropy).
* the label of a training frame is the cell of its Eq. 14 argmax direction.
* search: the C cells with the largest logits (ties -> lowest cell index) propose their
  children; the frame's direction is the argmax of Re{D_q Z} (Eq. 14) over those children
  (ties -> lowest index).  If the largest softmax probability is below theta the frame
  falls back to the exhaustive Eq. 14 argmax over every direction.
* training: Adam (Kingma & Ba, 2015, Algorithm 1) on the mean cross-entropy.

Parameter order, as flat FP32/FP64 vectors: W1 [H1][F], b1 [H1], W2 [H2][H1], b2 [H2],
W3 [C][H2], b3 [C] (row-major), F = 2K.
"""
from __future__ import annotations

import numpy as np

PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")
CELL_TIE = 1e-12


def child_cells(fine_dirs: np.ndarray, cell_dirs: np.ndarray) -> np.ndarray:
    """For every fine direction, the lowest index among the cell directions whose dot product
    with it is within CELL_TIE of the largest.  Directions are normalised first."""
    f = np.asarray(fine_dirs, dtype=np.float64)
    c = np.asarray(cell_dirs, dtype=np.float64)
    f = f / np.linalg.norm(f, axis=1, keepdims=True)
    c = c / np.linalg.norm(c, axis=1, keepdims=True)
    out = np.empty(f.shape[0], dtype=np.int64)
    for q in range(f.shape[0]):
        dots = c @ f[q]
        out[q] = int(np.flatnonzero(dots >= dots.max() - CELL_TIE)[0])
    return out


def children(cell_of: np.ndarray, n_cells: int) -> list[np.ndarray]:
    """The fine directions of every cell, ascending."""
    return [np.flatnonzero(cell_of == c) for c in range(n_cells)]


def features(Z: np.ndarray) -> np.ndarray:
    """x = interleaved (Re Z_k, Im Z_k) / ||Z|| per frame; 0 for a frame with ||Z|| = 0."""
    Z = np.asarray(Z, dtype=np.complex128)
    T, K = Z.shape
    x = np.empty((T, 2 * K))
    x[:, 0::2] = Z.real
    x[:, 1::2] = Z.imag
    n = np.sqrt(np.sum(x * x, axis=1))
    safe = np.where(n > 0, n, 1.0)
    return np.where(n[:, None] > 0, x / safe[:, None], 0.0)


def unflatten(theta: np.ndarray, F: int, H1: int, H2: int, C: int) -> dict:
    theta = np.asarray(theta, dtype=np.float64)
    shapes = [(H1, F), (H1,), (H2, H1), (H2,), (C, H2), (C,)]
    out, o = {}, 0
    for name, sh in zip(PARAM_NAMES, shapes):
        n = int(np.prod(sh))
        out[name] = theta[o:o + n].reshape(sh).copy()
        o += n
    assert o == theta.size, "parameter vector length does not match the layer sizes"
    return out


def flatten(params: dict) -> np.ndarray:
    return np.concatenate([np.asarray(params[n], dtype=np.float64).ravel() for n in PARAM_NAMES])


def round_bf16(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64: keep the top 16
    bits of the IEEE binary32 pattern after adding half of the dropped part's unit."""
    u = np.ascontiguousarray(np.asarray(a, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def forward(params: dict, x: np.ndarray, act_round=None) -> dict:
    """The network's forward pass in FP64.  ``act_round`` (e.g. ``round_bf16``) is applied to
    the input of every layer, modelling a kernel that stores activations in that type."""
    rnd = (lambda a: a) if act_round is None else act_round
    a0 = rnd(np.asarray(x, dtype=np.float64))
    z1 = a0 @ params["W1"].T + params["b1"]
    h1 = np.maximum(z1, 0.0)
    a1 = rnd(h1)
    z2 = a1 @ params["W2"].T + params["b2"]
    h2 = np.maximum(z2, 0.0)
    a2 = rnd(h2)
    logits = a2 @ params["W3"].T + params["b3"]
    return dict(a0=a0, z1=z1, a1=a1, z2=z2, a2=a2, logits=logits)


def softmax(logits: np.ndarray) -> np.ndarray:
    m = np.max(logits, axis=1, keepdims=True)
    e = np.exp(logits - m)
    return e / np.sum(e, axis=1, keepdims=True)


def loss_and_grads(params: dict, x: np.ndarray, labels: np.ndarray):
    """Mean cross-entropy and its gradient by the chain rule, layer by layer."""
    labels = np.asarray(labels, dtype=np.int64)
    n = x.shape[0]
    c = forward(params, x)
    p = softmax(c["logits"])
    loss = float(np.mean(-np.log(p[np.arange(n), labels])))
    g_logits = p.copy()
    g_logits[np.arange(n), labels] -= 1.0
    g_logits /= n
    g = {}
    g["W3"] = g_logits.T @ c["a2"]
    g["b3"] = np.sum(g_logits, axis=0)
    g_h2 = g_logits @ params["W3"]
    g_z2 = g_h2 * (c["z2"] > 0)
    g["W2"] = g_z2.T @ c["a1"]
    g["b2"] = np.sum(g_z2, axis=0)
    g_h1 = g_z2 @ params["W2"]
    g_z1 = g_h1 * (c["z1"] > 0)
    g["W1"] = g_z1.T @ c["a0"]
    g["b1"] = np.sum(g_z1, axis=0)
    return loss, g


def adam_step(params: dict, grads: dict, state: dict, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8) -> None:
    """One Adam update in place (Kingma & Ba, 2015, Algorithm 1); ``state`` holds m, v, t."""
    t = state.get("t", 0) + 1
    state["t"] = t
    for name in PARAM_NAMES:
        m = state.setdefault("m_" + name, np.zeros_like(params[name]))
        v = state.setdefault("v_" + name, np.zeros_like(params[name]))
        g = grads[name]
        m[...] = beta1 * m + (1.0 - beta1) * g
        v[...] = beta2 * v + (1.0 - beta2) * g * g
        mhat = m / (1.0 - beta1 ** t)
        vhat = v / (1.0 - beta2 ** t)
        params[name] = params[name] - lr * mhat / (np.sqrt(vhat) + eps)


def top_cells(logits: np.ndarray, n: int) -> np.ndarray:
    """The n largest logits per frame, largest first (ties -> lowest cell index)."""
    order = np.lexsort((np.broadcast_to(np.arange(logits.shape[1]), logits.shape), -logits), axis=1)
    return order[:, :n]


def learned_search(D: np.ndarray, Z: np.ndarray, logits: np.ndarray, kids: list, n_top: int, theta: float):
    """The proposal search: returns (direction index, score Re{D_q Z}, fell back?) per frame."""
    D = np.asarray(D, dtype=np.complex128)
    Z = np.asarray(Z, dtype=np.complex128)
    p = softmax(logits)
    conf = np.max(p, axis=1)
    cells = top_cells(logits, n_top)
    T = Z.shape[0]
    idx = np.empty(T, dtype=np.int64)
    best = np.empty(T)
    fb = conf < theta
    for t in range(T):
        if fb[t]:
            cand = np.arange(D.shape[0])
        else:
            cand = np.sort(np.concatenate([kids[c] for c in cells[t]]))
        y = (D[cand] @ Z[t]).real
        i = int(np.argmax(y))                      # first maximum = lowest index (cand ascending)
        idx[t] = cand[i]
        best[t] = y[i]
    return idx, best, fb
