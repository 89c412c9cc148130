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


def _wide_stream(T=300):
    """A stream whose basis is too wide for the tensor-core plan: 8 mics in a 15 cm-radius ball,
    N = 512, Q = 642 gives K = 181 (2K = 362 > 288), so the batch runs it in FP32."""
    rng = np.random.default_rng([I.SEED_BASE + 9, 8])
    mic = I.array_random_ball(rng, 8, radius=0.15)
    src = I.random_directions(rng, T)[:, None, :]
    snr = rng.uniform(-5.0, 20.0, size=T)
    frames = I.plane_wave_frames(rng, mic, T, 512, 16000.0, 343.0, src, snr, "white")
    return dict(mic_xyz=mic, dirs=I.icosphere(3), N=512, fs=16000.0, c=343.0, delta=1e-5, frames=frames,
                src_dirs=src, snr_db=snr)


def _streams():
    if "s" not in _S:
        import __graft_entry__
        __graft_entry__.build()
        wls = I.batched_streams(12, Q_choices=(642, 2562), N_choices=(256, 512), T_range=(50, 400))
        wls.append(_wide_stream())
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
        ref_prec = "fp32" if 2 * b.K > 288 or b.steering.M > 16 else prec   # no tensor-core plan
        idx, score, proj = sp.localize(b, f, "svd_exhaustive", ref_prec)
        assert torch.equal(bt.idx[i], idx), i
        assert torch.equal(bt.proj[i], proj), i
        assert torch.equal(bt.score[i], score), i


def test_localize_batched_matches_and_agrees_with_oracle():
    wls, bases, frames = _streams()
    idx, score, proj = sp.localize_batched(bases, frames, "svd_exhaustive", "fp16")
    for i in range(len(bases)):
        ref_prec = "fp32" if 2 * bases[i].K > 288 else "fp16"
        ref = sp.localize(bases[i], frames[i], "svd_exhaustive", ref_prec)
        assert torch.equal(idx[i], ref[0]) and torch.equal(proj[i], ref[2])
    # every stream of at most 8 microphones (the wide FP32 one included) against the FP64 oracle:
    # the same class wherever the oracle's top-2 margin exceeds 1e-4, and >= 99.5 % class
    # agreement over the pooled frames of these streams
    same_all = []
    checked = [i for i, wl in enumerate(wls) if wl["mic_xyz"].shape[0] <= 8]
    assert any(2 * bases[i].K > 288 for i in checked)
    for i in checked:
        wl = wls[i]
        tau = O.tdoa_farfield(wl["mic_xyz"], wl["dirs"], wl["fs"], wl["c"])
        ob = O.svd_basis(O.steering(tau, wl["N"]), wl["delta"])
        Y = O.svd_scores(ob["D"], O.project(ob["V"], O.phat(wl["frames"])))
        cls = O.direction_classes(tau)
        ref, _ = O.argmax_lowest(Y)
        m = O.top2_margin(Y, cls)
        got = idx[i].cpu().numpy()
        assert bases[i].K == ob["K"]
        assert np.all(cls[got][m > 1e-4] == cls[ref][m > 1e-4]), i
        same_all.append(cls[got] == cls[ref])
    same_all = np.concatenate(same_all)
    assert len(same_all) >= 400
    assert np.mean(same_all) >= 0.995, np.mean(same_all)


def test_batch_mixes_tensor_core_and_fp32_streams():
    """A basis beyond the tensor-core plan (2K > 288) runs its stream in FP32 inside the same
    launch, with the same result as sp_localize in FP32."""
    wls, bases, frames = _streams()
    big = [i for i, b in enumerate(bases) if 2 * b.K > 288]
    small = [i for i, b in enumerate(bases) if 2 * b.K <= 288]
    assert big and small, "the streams must mix wide (FP32) and tensor-core bases"
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
    sel = [i for i, b in enumerate(bases) if 2 * b.K <= 288][:6]
    bt = sp.Batch([bases[i] for i in sel], [frames[i] for i in sel], mode, prec)
    bt.run()
    torch.cuda.synchronize()
    sp.check_status()
    for k, i in enumerate(sel):
        idx, score, proj = sp.localize(bases[i], frames[i], mode, prec)
        assert torch.equal(bt.idx[k], idx) and torch.equal(bt.score[k], score)


def test_localize_batched_waits_for_the_callers_stream():
    """Frames written by work still queued on the caller's stream (behind a long device-side
    delay) are what the batch localises: the plan's set-up and run are ordered after it."""
    wls, bases, frames = _streams()
    sel = [i for i, b in enumerate(bases) if 2 * b.K <= 288][:3]
    refs = [sp.localize(bases[i], frames[i], "svd_exhaustive", "fp16")[0] for i in sel]
    bufs = [torch.zeros_like(frames[i]) for i in sel]
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        torch.cuda._sleep(200_000_000)          # ~0.1 s of device time before the copies
        for buf, i in zip(bufs, sel):
            buf.copy_(frames[i])
        idx, _, _ = sp.localize_batched([bases[i] for i in sel], bufs, "svd_exhaustive", "fp16")
    torch.cuda.synchronize()
    for a, r in zip(idx, refs):
        assert torch.equal(a, r)


def _offset_copy(f):
    """A copy of f whose data starts 8 bytes off a 16-byte boundary (the register-fed GEMM1)."""
    flat = torch.empty(f.numel() + 1, dtype=f.dtype, device=f.device)
    v = flat[1:].view(f.shape)
    v.copy_(f)
    return v


def test_autotuned_plan_is_stored_and_reused(tmp_path):
    """An autotuned plan with a tune cache stores its shape under the batch's signature; a
    second plan for the same batch takes it from the file (no measurement) and gives the same
    results; another batch has another signature.  With the kernel choice tuned, a stream on
    the register-fed GEMM1 equals sp_localize on a buffer that takes that kernel."""
    import json
    wls, bases, frames = _streams()
    path = tmp_path / "tune.json"
    sp.set_tune_cache(path)
    try:
        b1 = sp.Batch(bases, frames, "svd_exhaustive", "fp16", autotune=True, tune_kernels=True)
        i1 = b1.info()
        assert not i1["from_cache"] and i1["ms"] > 0
        plans = json.loads(path.read_text())["plans"]
        assert len(plans) == 1
        (key, entry), = plans.items()
        assert key.endswith("/k")
        assert entry["branches"] == i1["branches"] and entry["tiles_per_cta"] == i1["tiles_per_cta"]
        assert entry["proj_variant"] == i1["proj_variant"]
        b2 = sp.Batch(bases, frames, "svd_exhaustive", "fp16", autotune=True, tune_kernels=True)
        i2 = b2.info()
        assert i2["from_cache"]
        assert all(i2[k] == i1[k] for k in ("branches", "tiles_per_cta", "proj_variant", "grouped"))
        b1.run()
        b2.run()
        torch.cuda.synchronize()
        sp.check_status()
        for i in range(len(bases)):
            assert torch.equal(b1.idx[i], b2.idx[i]) and torch.equal(b1.proj[i], b2.proj[i]), i
            b, f = bases[i], frames[i]
            if 2 * b.K > 288:
                continue
            ref = f
            if i1["proj_variant"] == 1 and b.steering.M == 7:
                ref = _offset_copy(f)
            idx, score, proj = sp.localize(b, ref, "svd_exhaustive", "fp16")
            assert torch.equal(b1.idx[i], idx) and torch.equal(b1.proj[i], proj), i
        b3 = sp.Batch(bases[:-1], frames[:-1], "svd_exhaustive", "fp16", autotune=True, tune_kernels=True)
        assert not b3.info()["from_cache"]
        assert len(json.loads(path.read_text())["plans"]) == 2
        b4 = sp.Batch(bases, frames, "svd_exhaustive", "fp16", autotune=True)   # no kernel choice: own key
        assert not b4.info()["from_cache"] and b4.info()["proj_variant"] == 0
    finally:
        sp.set_tune_cache(None)


def _shared_basis_streams():
    """Nine streams cut from the first three streams' frames (three slices each, so three per
    basis: the plan forms three groups), plus one 8-byte-offset copy that stays alone."""
    wls, bases, frames = _streams()
    sb, sf = [], []
    for i in range(3):
        f = frames[i]
        T = f.shape[0]
        for a, z in [(0, T // 3), (T // 3, T // 2), (T // 2, T)]:
            sb.append(bases[i])
            sf.append(f[a:z].clone())
    sb.append(bases[0])
    sf.append(_offset_copy(frames[0][:40]))
    return sb, sf


@pytest.mark.parametrize("mode,prec,autotune", [("svd_exhaustive", "fp16", False), ("svd_exhaustive", "fp16", True),
                                                ("svd_exhaustive", "fp32", False), ("svd_kdtree", "fp16", False)])
def test_grouped_plan_equals_per_stream_localize(mode, prec, autotune):
    """Streams that share a basis are copied into one buffer and localised by one call; each
    stream's idx, score and proj are bit-identical to its own sp_localize call (the unaligned
    stream runs alone, as sp_localize runs it on the register-fed kernel)."""
    sb, sf = _shared_basis_streams()
    bt = sp.Batch(sb, sf, mode, prec, autotune=autotune, group=not autotune)
    info = bt.info()
    assert info["n_groups"] == 3
    if not autotune:
        assert info["grouped"]
    for f in bt.idx:
        f.fill_(-7)
    bt.run()
    torch.cuda.synchronize()
    sp.check_status()
    for i, (b, f) in enumerate(zip(sb, sf)):
        ref_prec = "fp32" if 2 * b.K > 288 or b.steering.M > 16 else prec
        idx, score, proj = sp.localize(b, f, mode, ref_prec)
        assert torch.equal(bt.idx[i], idx), i
        assert torch.equal(bt.score[i], score), i
        assert torch.equal(bt.proj[i], proj), i
