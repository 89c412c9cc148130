"""The batched form: many streams with different arrays, grids, N and frame counts in one
CUDA-graph launch give exactly the per-stream results of sp_localize (same kernels), and
those agree with the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1811_11785_gb300 as sp
from paper_1811_11785_gb300 import inputs as I

pytestmark = pytest.mark.gpu

_S = {}


def _streams():
    if "s" not in _S:
        import __graft_entry__
        __graft_entry__.build()
        wls = I.batched_streams(12, Q_choices=(642, 2562), N_choices=(256, 512), T_range=(50, 400))
        bases, frames = [], []
        for wl in wls:
            st = sp.build_steering(wl["mic_xyz"], wl["dirs"], wl["fs"], wl["c"], wl["N"])
            bases.append(sp.svd_reduce(st, wl["delta"]))
            frames.append(torch.from_numpy(wl["frames"]).cuda())
        _S["s"] = (wls, bases, frames)
    return _S["s"]


@pytest.mark.parametrize("prec", ["fp16", "fp32"])
@pytest.mark.parametrize("autotune", [False, True])
def test_batch_equals_per_stream_localize(prec, autotune):
    wls, bases, frames = _streams()
    bt = sp.Batch(bases, frames, "svd_exhaustive", prec, autotune=autotune)
    for f in bt.idx:
        f.fill_(-7)
    bt.run()
    torch.cuda.synchronize()
    sp.check_status()
    info = bt.info()
    assert info["branches"] >= 1 and info["tiles_per_cta"] in (1, 2, 4)
    if autotune:
        assert info["ms"] > 0
    for i, (b, f) in enumerate(zip(bases, frames)):
        ref_prec = "fp32" if 2 * b.K > 320 or b.steering.M > 16 else prec   # no tensor-core plan
        idx, score, proj = sp.localize(b, f, "svd_exhaustive", ref_prec)
        assert torch.equal(bt.idx[i], idx), i
        assert torch.equal(bt.proj[i], proj), i
        assert torch.equal(bt.score[i], score), i


def test_localize_batched_matches_and_agrees_with_oracle():
    wls, bases, frames = _streams()
    idx, score, proj = sp.localize_batched(bases, frames, "svd_exhaustive", "fp16")
    for i in range(len(bases)):
        ref_prec = "fp32" if 2 * bases[i].K > 320 else "fp16"
        ref = sp.localize(bases[i], frames[i], "svd_exhaustive", ref_prec)
        assert torch.equal(idx[i], ref[0]) and torch.equal(proj[i], ref[2])
    Ms = [wl["mic_xyz"].shape[0] for wl in wls]
    for i in sorted(range(len(wls)), key=lambda j: Ms[j])[:3]:     # the three smallest arrays
        wl = wls[i]
        tau = O.tdoa_farfield(wl["mic_xyz"], wl["dirs"], wl["fs"], wl["c"])
        ob = O.svd_basis(O.steering(tau, wl["N"]), wl["delta"])
        Y = O.svd_scores(ob["D"], O.project(ob["V"], O.phat(wl["frames"])))
        cls = O.direction_classes(tau)
        ref, _ = O.argmax_lowest(Y)
        m = O.top2_margin(Y, cls)
        got = idx[i].cpu().numpy()
        assert bases[i].K == ob["K"]
        assert np.all(cls[got][m > 1e-4] == cls[ref][m > 1e-4])


def test_batch_mixes_tensor_core_and_fp32_streams():
    """A basis beyond the tensor-core plan (2K > 320) runs its stream in FP32 inside the same
    launch, with the same result as sp_localize in FP32."""
    wls, bases, frames = _streams()
    big = [i for i, b in enumerate(bases) if 2 * b.K > 320]
    small = [i for i, b in enumerate(bases) if 2 * b.K <= 320]
    if not big or not small:
        pytest.skip("the seeded streams hold no mix of large and small ranks")
    sel = big[:2] + small[:2]
    bt = sp.Batch([bases[i] for i in sel], [frames[i] for i in sel], "svd_exhaustive", "fp16")
    bt.run()
    torch.cuda.synchronize()
    assert bt.info()["n_fp32"] == len(big[:2])
    for k, i in enumerate(sel):
        prec = "fp32" if i in big else "fp16"
        ref = sp.localize(bases[i], frames[i], "svd_exhaustive", prec)
        assert torch.equal(bt.idx[k], ref[0])


@pytest.mark.parametrize("mode,prec", [("svd_kdtree", "fp16"), ("svd_exhaustive", "bf16")])
def test_batch_other_modes_equal_per_stream(mode, prec):
    wls, bases, frames = _streams()
    sel = [i for i, b in enumerate(bases) if 2 * b.K <= 320][:6]
    bt = sp.Batch([bases[i] for i in sel], [frames[i] for i in sel], mode, prec)
    bt.run()
    torch.cuda.synchronize()
    sp.check_status()
    for k, i in enumerate(sel):
        idx, score, proj = sp.localize(bases[i], frames[i], mode, prec)
        assert torch.equal(bt.idx[k], idx) and torch.equal(bt.score[k], score)
