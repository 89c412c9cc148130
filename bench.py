"""Benchmark of the SVD-PHAT hot path on GB300.

Workload: 7-mic planar array (centre + 6 mics on a 5 cm circle), fs 16 kHz, N = 512 (Hann,
B = 257 bins), Q = 2562 icosphere directions, K from delta = 1e-5 (K = 48), 65,536 frames
per step with one white-noise plane-wave source per frame at SNR U(-5, 20) dB (synthetic).
A step is one pass of Algorithm 1's online path over the batch: PHAT -> Z = V^H X ->
exhaustive Re{D Z} argmax (FP16 tensor cores, then FP32 rescoring of every class within the
FP16 rounding bound of the best; frames with more than 14 such classes go to an FP32 scan
over every class on a device list, empty on this workload) -> Y_qbar from the row of W
(online step 4): five kernel launches (GEMM1, scan, list scan, list finalize, step 4) and a
4-byte reset of the list count.  The STFT batch (943 MB) is larger than L2, so no flush is
needed.

Extra keys (unless --no-extras): the same frames through FP32 SRP-PHAT, the FP32 / BF16
paths and the k-d tree; the 3-D 7-mic array with Q = 10242 (exhaustive, learned proposal,
k-d tree on 2^20 frames); 256 batched streams in one CUDA-graph launch.  --only c5 (opt-in,
minutes of basis set-up): the 16-mic, N = 1024 array on the level-6 grid (Q = 40,962).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--prec fp16|bf16]
                [--frames T] [--no-extras] [--only array3d|batched|batched_default|c5|samples|sweep|kdtree] [--array3d-frames T]
Under torchrun each rank localises its own 65,536 frames (weak scaling, no collective on the
data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "planar_q2562"
METRIC = "localized frames/s at >=99.5% argmax agreement vs FP64 oracle"
UNIT = "frames/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# DRAM bytes read + written per frame by the dominant kernel (svd_proj_tma_kernel), from one
# ncu capture of this version of the kernel on 19,456 frames of the same workload, scaled to a
# launch by the frame count (traffic grows in proportion to frames).  None until captured.
TRAFFIC_PER_FRAME = 16121.7     # 313,662,976 B / 19,456 frames (read 307.7 MB, write 5.9 MB)
DOMINANT_KERNEL = "svd_proj_tma_kernel"


def _peaks():
    try:
        p = json.load(open(PEAKS_FILE))
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """Samples nvidia-smi every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        loaded = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        out.update(sm_mhz=statistics.median(loaded) if loaded else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=sorted(reasons), samples=len(rows))
        return out


def _oracle_block(args):
    """One process's share of the FP64 oracle sample: PHAT, Z = V^H X, Re{D Z}, the argmax and
    online step 4 (Algorithm 1) for a block of frames.  Returns (idx, Y)."""
    import oracle as O
    fr, V, D, tau, N = args
    X = O.phat(fr)
    Y = O.svd_scores(D, O.project(V, X))
    idx, _ = O.argmax_lowest(Y)
    O.score_row(tau, idx, X, N)
    return idx, Y


def _oracle_step4(args):
    """Online step 4 of the oracle for given indices (error statistics, not timed)."""
    import oracle as O
    fr, tau, idx, N = args
    return O.score_row(tau, idx, O.phat(fr), N)


def _noop(_):
    return 0


_POOL = None


def oracle_pool():
    """A pool of spawned processes, one per host core the job may use, each with one BLAS thread:
    the oracle's per-frame work runs on every core (frames are independent)."""
    global _POOL
    if _POOL is None:
        import multiprocessing as mp
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[v] = "1"
        _POOL = mp.get_context("spawn").Pool(_cores())
        _POOL.map(_noop, range(2 * _cores()))   # start every worker before any timing
    return _POOL


def oracle_sample(wl, n_frames: int, seed: int = 7):
    """FP64 oracle on a bounded sample of the workload, the frames split over every host core:
    returns (frames/s, seconds, sel, idx_ref, Y, cls)."""
    import oracle as O
    tau = O.tdoa_farfield(wl["mic_xyz"], wl["dirs"], wl["fs"], wl["c"])
    W = O.steering(tau, wl["N"])
    ob = O.svd_basis(W, wl["delta"])            # offline (Algorithm 1 offline steps), not timed
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(wl["frames"].shape[0], n_frames, replace=False))
    fr = wl["frames"][sel]
    pool = oracle_pool()
    blocks = np.array_split(np.arange(n_frames), _cores())
    args = [(fr[b], ob["V"], ob["D"], tau, wl["N"]) for b in blocks if len(b)]
    t0 = time.perf_counter()
    res = pool.map(_oracle_block, args)
    dt = time.perf_counter() - t0
    idx = np.concatenate([r[0] for r in res])
    Y = np.concatenate([r[1] for r in res])
    oracle_sample.last = dict(tau=tau, fr=fr, L=W.shape[1], blocks=[b for b in blocks if len(b)])
    return n_frames / dt, dt, sel, idx, Y, O.direction_classes(tau)


def oracle_step4(gi, N):
    """The oracle's online step-4 scores of the last sample for the indices gi (untimed)."""
    last = oracle_sample.last
    res = oracle_pool().map(_oracle_step4, [(last["fr"][b], last["tau"], gi[b], N) for b in last["blocks"]])
    return np.concatenate(res)


def arm_config(K: int, T: int) -> dict:
    """The config of the measured workload, the same for both arms."""
    return {"workload": f"{WORKLOAD}: 7-mic planar array, Q=2562, N=512, K={K}, "
                        f"{T} frames/step/GPU, SNR U(-5,20) dB",
            "frames_per_step": T, "Q": 2562, "M": 7, "N": 512, "K": K,
            "mode": "svd_exhaustive (FP16/BF16 scan + FP32 rescoring of every class within the "
                    "rounding bound) + online step 4",
            "l2": "inputs (943 MB STFT) larger than L2; no flush"}


def clocks_sm_mhz(clk) -> float | None:
    """The median SM clock the Clocks sampler saw, if any."""
    try:
        return float(clk["sm_mhz"]) if clk and clk.get("sm_mhz") else None
    except Exception:
        return None


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    """The oracle arm: the FP64 CPU oracle on the same workload, bounded samples per step."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from paper_1811_11785_gb300 import inputs as I
    wl = I.workload(WORKLOAD, T=8192)
    n = 1024
    for _ in range(args.warmup):
        oracle_sample(wl, 256)
    rates, secs = [], []
    for s in range(args.steps):
        r, dt, *_ = oracle_sample(wl, n, seed=100 + s)
        rates.append(r)
        secs.append(dt)
    import oracle as O
    tau = O.tdoa_farfield(wl["mic_xyz"], wl["dirs"], wl["fs"], wl["c"])
    K = O.svd_basis(O.steering(tau, wl["N"]), wl["delta"])["K"]
    v = n * len(secs) / sum(secs)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(secs) / len(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": arm_config(K, args.frames),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": _cores(), "kind": "oracle",
                             "sample": f"{n} frames per step drawn from an 8192-frame batch of the workload, FP64, "
                                       f"split over {_cores()} spawned processes with one BLAS thread each"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def kdtree_stats(sp, b, frames, torch, reps=3):
    """The k-d tree search alone (sp_kdtree_search on sp_project's Z): mean nodes and leaf
    buckets visited per query, and the bytes those visits read (leaf points 2K x 32 floats and
    32 indices per bucket, 16 bytes per node, the query) per second of the search."""
    Z = sp.project(b, frames, "fp16")
    _, _, vis = sp.kdtree_search(b, Z)
    torch.cuda.synchronize()
    qps = _rate(lambda: sp.kdtree_search(b, Z, visits=False), reps, frames.shape[0], torch)
    T = frames.shape[0]
    v = vis.double().mean(dim=0).tolist()
    K = b.K
    bytes_per_q = v[1] * (2 * K * 32 * 4 + 32 * 4) + v[0] * 16 + 2 * K * 4
    info = b.kdtree_info()
    return {"queries_per_s": qps, "nodes_visited_mean": v[0], "leaf_buckets_visited_mean": v[1],
            "leaf_buckets_total": (info["n_nodes"] + 1) // 2, "nodes_total": info["n_nodes"],
            "points_visited_mean": 32 * v[1], "l2_read_GBps": bytes_per_q * qps / 1e9,
            "bytes_read_per_query": bytes_per_q}


def bench_kdtree(sp, I, torch, T=32768):
    """The k-d tree search alone on the 3-D 7-microphone array, Q = 10242 (level-5 grid), K = 71:
    T frames of 1-2 white sources in isotropic noise (the array3d_q10242 workload), projected by
    sp_project, then sp_kdtree_search with its visit statistics."""
    wl = I.workload("array3d_q10242", T=T, seed_offset=11)
    st = sp.build_steering(wl["mic_xyz"], wl["dirs"], wl["fs"], wl["c"], wl["N"])
    b = sp.svd_reduce(st, wl["delta"])
    frames = torch.from_numpy(wl["frames"]).cuda()
    out = kdtree_stats(sp, b, frames, torch)
    out["workload"] = f"array3d_q10242: 7-mic 3-D array, Q=10242, N=512, K={b.K}, {T} frames"
    return out


C4_UNIQUE, C4_REPEAT = 32768, 32
LEARNED_N_TOP, LEARNED_THETA = 8, 0.2


def bench_array3d(sp, I, torch, unique=C4_UNIQUE, repeat=C4_REPEAT):
    """The k-d tree and learned-proposal forms on the 3-D 7-mic array, Q = 10242 (level-5
    grid), K = 71: 1,048,576 frames per pass (32,768 unique frames of 1-2 white sources in
    isotropic noise at 0-20 dB, repeated 32 times on the device).  The proposal (level-3
    cells, 2K -> 256 -> 256 -> 642) is trained first, untimed, on 65,536 frames of 1-3
    sources the method labels itself."""
    wl = I.workload("array3d_q10242", T=unique, seed_offset=11)
    st = sp.build_steering(wl["mic_xyz"], wl["dirs"], wl["fs"], wl["c"], wl["N"])
    b = sp.svd_reduce(st, wl["delta"])
    uniq = torch.from_numpy(wl["frames"]).cuda()
    frames = uniq.repeat(repeat, 1, 1) if repeat > 1 else uniq
    T = frames.shape[0]
    rng = np.random.default_rng(I.SEED_BASE + 50)
    tr, _, _ = I.training_frames(rng, wl["mic_xyz"], 65536, wl["N"], wl["fs"], wl["c"])
    p = sp.Proposal(b, I.icosphere(3), seed=5)
    x, y = p.examples(torch.from_numpy(tr).cuda(), "fp16")
    t0 = time.perf_counter()
    losses = p.train(x, y, epochs=6, batch=512, lr=1e-3, seed=6)
    train_s = time.perf_counter() - t0
    del x, y, tr

    def rate(fn, n):
        return _rate(fn, n, T, torch)

    ex = sp.localize(b, uniq, "svd_exhaustive", "fp16", score=False)[0]
    li, _, _, fb = p.localize(uniq, "fp16", n_top=LEARNED_N_TOP, theta=LEARNED_THETA, score=False)
    kd = sp.localize(b, uniq, "svd_kdtree", "fp16", score=False)[0]
    torch.cuda.synchronize()
    # per-stage times (ms per pass of T frames)
    Z = sp.project(b, frames, "fp16")
    zn2 = (Z.real ** 2 + Z.imag ** 2).sum(dim=1).float()
    ms = lambda fn, n: T / rate(fn, n) * 1000
    t_proj = ms(lambda: sp.project(b, frames, "fp16"), 3)
    t_mlp = ms(lambda: p.infer(Z, zn2), 3)
    t_exh = ms(lambda: sp.localize(b, frames, "svd_exhaustive", "fp16"), 3)
    t_exh_ns = ms(lambda: sp.localize(b, frames, "svd_exhaustive", "fp16", score=False), 3)
    t_lrn = ms(lambda: p.localize(frames, "fp16", n_top=LEARNED_N_TOP, theta=LEARNED_THETA, fallback=False), 3)
    t_lrn_ns = ms(lambda: p.localize(frames, "fp16", n_top=LEARNED_N_TOP, theta=LEARNED_THETA, score=False,
                                     fallback=False), 3)
    t_kd = ms(lambda: sp.localize(b, frames, "svd_kdtree", "fp16"), 1)
    del Z, zn2
    out = {
        "workload": f"array3d_q10242: 7-mic 3-D array, Q=10242, N=512, K={b.K}, {T} frames per pass "
                    f"({unique} unique x {repeat}), 1-2 sources, isotropic noise 0-20 dB",
        "svd_exhaustive_fp16_frames_per_s": T / t_exh * 1000,
        "svd_learned_fp16_frames_per_s": T / t_lrn * 1000,
        "svd_kdtree_fp16_frames_per_s": T / t_kd * 1000,
        "ms_per_pass": {"gemm1": t_proj, "exhaustive_scan": t_exh_ns - t_proj,
                        "mlp_tc_kernel": t_mlp, "rescore_and_fallback_scan": t_lrn_ns - t_proj - t_mlp,
                        "step4_bulk_kernel": t_exh - t_exh_ns, "kdtree": t_kd - (t_exh - t_exh_ns) - t_proj},
        "learned": {"n_top": LEARNED_N_TOP, "theta": LEARNED_THETA, "cells": 642, "hidden": [256, 256],
                    "train_frames": 65536, "epochs": 6, "train_s": train_s,
                    "final_loss": float(losses[-1]),
                    "fallback_fraction": float(fb.float().mean()),
                    "agreement_vs_exhaustive": float((li == ex).float().mean())},
        "kdtree_agreement_vs_exhaustive": float((kd == ex).float().mean()),
        "kdtree_search": kdtree_stats(sp, b, uniq, torch),
    }
    return out


C5_FRAMES, C5_TRAIN, C5_CHUNK, C5_EPOCHS, C5_ORACLE = 65536, 1 << 21, 65536, 3, 256
C5_N_TOP = (2, 4)    # cells of ~64 children: at most 512 candidates per frame (8 cells overflow it)


def _oracle_srp_block(args):
    """FP64 SRP-PHAT (Eq. 5, 9: Re{W X} with W from Eq. 4, 8 and X from Eq. 3, 7) of a frame
    sample over a block of directions, W built 256 rows at a time.  Returns Y [frames][block]."""
    import oracle as O
    fr, tau, N = args
    X = O.phat(fr)
    out = np.empty((fr.shape[0], tau.shape[0]))
    for q0 in range(0, tau.shape[0], 256):
        out[:, q0:q0 + 256] = O.srp_scores(O.steering(tau[q0:q0 + 256], N), X)
    return out


def bench_c5(sp, I, torch):
    """The 16-mic array in a 5 cm-radius ball (the one of the ball16_n1024_q642 parity
    cases), N = 1024 (B = 513, P = 120, L = 61,560), on the level-6 grid (Q = 40,962): the
    exhaustive FP16 path and the learned proposal (level-3 cells, top-4 cells of ~64
    children each) on 65,536 reverberant frames per pass (1-3 white sources with exponential
    tails, T60 0.2-0.6 s, white noise at -5..20 dB, drawn on the device).  The proposal trains
    on 2^21 frames of the same generator (other seeds).  The FP64 oracle's SRP-PHAT (Eq. 5)
    scores a 256-frame sample over all 40,962 directions on every host core (the section's
    cpu_baseline); both searches are compared with its argmax on that sample."""
    import oracle as O
    fs, c, N = 16000.0, 343.0, 1024
    mic = I.array_random_ball(np.random.default_rng([I.SEED_BASE + 7, 4]), 16)
    dirs = I.icosphere(6)
    t0 = time.perf_counter()
    st = sp.build_steering(mic, dirs, fs, c, N)
    b = sp.svd_reduce(st, 1e-5)
    torch.cuda.synchronize()
    basis_s = time.perf_counter() - t0
    frames, _, n_src = I.reverberant_frames_gpu(I.SEED_BASE + 60, mic, C5_FRAMES, N, fs, c)
    T = frames.shape[0]
    p = sp.Proposal(b, I.icosphere(3), seed=5)
    t1 = time.perf_counter()
    x = torch.empty((C5_TRAIN, p.F), dtype=torch.float32, device="cuda")
    y = torch.empty(C5_TRAIN, dtype=torch.int32, device="cuda")
    for i, r0 in enumerate(range(0, C5_TRAIN, C5_CHUNK)):
        tr, _, _ = I.reverberant_frames_gpu(I.SEED_BASE + 1000 + i, mic, C5_CHUNK, N, fs, c)
        x[r0:r0 + C5_CHUNK], y[r0:r0 + C5_CHUNK] = p.examples(tr, "fp16")
        del tr
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t1
    t1 = time.perf_counter()
    losses = p.train(x, y, epochs=C5_EPOCHS, batch=1024, lr=1e-3, seed=6)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    del x, y

    ex16, _, pr16 = sp.localize(b, frames, "svd_exhaustive", "fp16", score=False)
    ex32 = sp.localize(b, frames, "svd_exhaustive", "fp32", score=False)[0]
    res = {}
    for nt in C5_N_TOP:
        li, _, _, fb = p.localize(frames, "fp16", n_top=nt, theta=LEARNED_THETA, score=False)
        res[nt] = (li, fb)
    torch.cuda.synchronize()
    ms = lambda fn, n: T / _rate(fn, n, T, torch) * 1000
    t_proj = ms(lambda: sp.project(b, frames, "fp16"), 3)
    t_exh = ms(lambda: sp.localize(b, frames, "svd_exhaustive", "fp16"), 3)
    t_exh_ns = ms(lambda: sp.localize(b, frames, "svd_exhaustive", "fp16", score=False), 3)
    t_lrn = {nt: ms(lambda: p.localize(frames, "fp16", n_top=nt, theta=LEARNED_THETA, fallback=False), 3)
             for nt in C5_N_TOP}

    # FP64 SRP-PHAT on a sample, every host core (the section's cpu_baseline)
    rng = np.random.default_rng(I.SEED_BASE + 62)
    sel = np.sort(rng.choice(T, C5_ORACLE, replace=False))
    fr_s = frames[torch.from_numpy(sel).cuda()].cpu().numpy()
    tau = O.tdoa_farfield(mic, dirs, fs, c)
    pool = oracle_pool()
    blocks = np.array_split(np.arange(tau.shape[0]), 2 * _cores())
    t2 = time.perf_counter()
    Y = np.concatenate(pool.map(_oracle_srp_block, [(fr_s, tau[bl], N) for bl in blocks]), axis=1)
    oracle_s = time.perf_counter() - t2
    ref, ymax = O.argmax_lowest(Y)
    cls = O.direction_classes(tau)
    L = st.L
    unit = dirs / np.linalg.norm(dirs, axis=1, keepdims=True)

    def vs_fp64(idx):
        # on a 1-degree grid the runner-up is often a neighbour within 1e-4 L of the best, so
        # besides the same-direction rate report the SRP-PHAT energy given up and the angle
        i = idx.cpu().numpy()[sel]
        same = cls[i] == cls[ref]
        loss = (ymax - Y[np.arange(len(sel)), i]) / L
        ang = np.degrees(np.arccos(np.clip(np.sum(unit[i] * unit[ref], axis=1), -1.0, 1.0)))
        q = lambda v: {"median": float(np.median(v)), "p99": float(np.quantile(v, 0.99)), "max": float(v.max())}
        return {"agreement": float(same.mean()), "energy_loss_over_L": q(loss), "angle_deg": q(ang)}

    learned = {}
    for nt in C5_N_TOP:
        li, fb = res[nt]
        learned[f"n_top_{nt}"] = {
            "frames_per_s": T / t_lrn[nt] * 1000, "ms_per_pass": t_lrn[nt],
            "fallback_fraction": float(fb.float().mean()),
            "agreement_vs_exhaustive_fp16": float((li == ex16).float().mean()),
            "vs_fp64_srp_phat": vs_fp64(li)}
    return {
        "workload": f"ball16_n1024_q40962: 16-mic array in a 5 cm-radius ball, N=1024, Q=40962, K={b.K}, "
                    f"{T} frames per pass, 1-3 white sources with exponential reverberant tails "
                    f"(T60 U(0.2, 0.6) s), white noise -5..20 dB",
        "svd_exhaustive_fp16_frames_per_s": T / t_exh * 1000,
        "ms_per_pass": {"gemm1": t_proj, "exhaustive_scan": t_exh_ns - t_proj, "step4": t_exh - t_exh_ns},
        "gemm1_tflops": 2.0 * T * 2 * L * 2 * b.K / (t_proj * 1e-3) / 1e12,
        "fp16_agreement_vs_fp32_path": float((ex16 == ex32).float().mean()),
        "exhaustive_fp16_vs_fp64_srp_phat": vs_fp64(ex16),
        "fp64_sample": {"frames": C5_ORACLE,
                        "sources_per_frame": np.bincount(n_src.cpu().numpy()[sel], minlength=4)[1:].tolist()},
        "learned": {"theta": LEARNED_THETA, "cells": p.C, "train_frames": C5_TRAIN, "epochs": C5_EPOCHS,
                    "batch": 1024, "generate_and_label_s": gen_s, "train_s": train_s,
                    "loss_per_epoch": [float(v) for v in losses], **learned},
        "cpu_baseline": {"value": C5_ORACLE / oracle_s, "unit": "frames/s", "cores": _cores(), "kind": "oracle",
                         "sample": f"FP64 SRP-PHAT (Eq. 5) of {C5_ORACLE} frames over all {tau.shape[0]} directions"},
        "basis_setup_s": basis_s,
    }


def bench_samples(sp, I, torch, T=65536, seg_frames=1024):
    """Localisation from time samples (Section 2's STFT front end, then Algorithm 1's online
    path): the planar 7-microphone array, Q = 2562, N = 512, hop 256, T frames from
    T * 256 + 256 samples per microphone (float32, channel rows), one white source per segment of
    seg_frames frames from a seeded direction, white noise at 10 dB.  Reports frames/s through
    sp_localize_samples (algorithmic bytes: the 7 x 256 new samples of a frame, 7,168 B), the
    STFT kernel alone against the HBM peak (reads 7,168 B, writes 14,392 B per frame), and the
    same with a binary mask keeping half the bins."""
    wl = I.workload(WORKLOAD, T=64)
    N, hop = 512, 256
    st = sp.build_steering(wl["mic_xyz"], wl["dirs"], wl["fs"], wl["c"], N)
    b = sp.svd_reduce(st, wl["delta"])
    rng = np.random.default_rng(I.SEED_BASE + 80)
    seg = seg_frames * hop
    n_seg = (T * hop + hop + seg - 1) // seg
    x = np.concatenate([I.time_signals(rng, wl["mic_xyz"], seg, wl["fs"], wl["c"], u, 10.0)
                        for u in I.random_directions(rng, n_seg)], axis=1)[:, :T * hop + hop]
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    del x
    assert sp.n_frames(xt.shape[1], N, hop) == T
    out = (torch.empty(T, dtype=torch.int32, device="cuda"), torch.empty(T, dtype=torch.float32, device="cuda"),
           torch.empty(T, dtype=torch.float32, device="cuda"))
    frames = torch.empty((T, 7, N // 2 + 1), dtype=torch.complex64, device="cuda")
    mask = torch.from_numpy(I.random_mask(rng, T, N // 2 + 1, 0.5)).cuda()
    peak, peak_kind = _peaks()

    def stft_only():
        rc = sp.lib().sp_stft(ctypes.c_void_p(xt.data_ptr()), 7, xt.shape[1], xt.stride(0), N, hop, None,
                              ctypes.c_void_p(frames.data_ptr()), None,
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0, sp.lib().sp_last_error()

    r_all = _rate(lambda: sp.localize_samples(b, xt, hop, "svd_exhaustive", "fp16", T=T, out=out), 10, T, torch)
    r_mask = _rate(lambda: sp.localize_samples(b, xt, hop, "svd_exhaustive", "fp16", mask=mask, T=T, out=out), 10,
                   T, torch)
    r_stft = _rate(stft_only, 10, T, torch)
    stft_gbs = r_stft * (7 * hop * 4 + 7 * (N // 2 + 1) * 8) / 1e9
    return {"workload": f"planar_q2562 from time samples: 7 mics, N={N}, hop={hop}, K={b.K}, {T} frames "
                        f"({T * hop + hop} samples per microphone, float32), one white source per {seg_frames} "
                        "frames, white noise 10 dB",
            "frames_per_s": r_all, "algorithmic_bytes_per_frame": 7 * hop * 4,
            "sample_GBps": r_all * 7 * hop * 4 / 1e9,
            "masked_half_bins_frames_per_s": r_mask,
            "stft_kernel": {"frames_per_s": r_stft, "GBps": stft_gbs, "peak": peak, "peak_source": peak_kind,
                            "frac": stft_gbs / peak,
                            "bytes_per_frame": 7 * hop * 4 + 7 * (N // 2 + 1) * 8}}


SWEEP_DELTAS = (1e-7, 1e-6, 1e-5, 1e-4, 1e-3, 1e-2, 1e-1)


def bench_delta_sweep(sp, I, torch, n_cfg=12, seconds=1.0):
    """Section 4's experiment on synthetic rooms: for the 1-D, 2-D and 3-D arrays of Table 2
    (Table 1: fs 16 kHz, c 343 m/s, N 256, hop 128, Q 2562), n_cfg shoebox configurations
    (10 x 10 x 3 m, wall reflection coefficients U(0.2, 0.5), image method to 2 reflections, a
    white-noise source, white noise at 0-30 dB; TIMIT is not available), each `seconds` of
    audio through the STFT front end.  Per delta: K (Eq. 11), the gain Q/K, and Delta RMSE, the
    mean over configurations of the energy-weighted DOA error (Eq. 20) of SVD-PHAT (FP32
    exhaustive search) minus that of SRP-PHAT on the same frames."""
    fs, c, N, hop = 16000.0, 343.0, 256, 128
    dirs = I.icosphere(4)
    arrays = {1: ("1-D linear", I.array_linear_1d()), 2: ("2-D planar", I.array_planar_2d_table()),
              3: ("3-D", I.array_3d())}
    out = {"workload": f"{n_cfg} shoebox rooms per array, {seconds:.1f} s of audio each, N={N}, hop={hop}, Q=2562",
           "deltas": list(SWEEP_DELTAS)}
    t0 = time.perf_counter()
    for alpha, (name, mic) in arrays.items():
        st = sp.build_steering(mic, dirs, fs, c, N, materialize_w=True)
        bases = [sp.svd_reduce(st, d) for d in SWEEP_DELTAS]
        rng = np.random.default_rng(I.SEED_BASE + 90 + alpha)
        r_srp, r_svd = [], [[] for _ in SWEEP_DELTAS]
        for _ in range(n_cfg):
            x, s0, _, _ = I.room_signals(rng, mic, int(seconds * fs), fs, c)
            frames = sp.stft(torch.from_numpy(x).cuda(), N, hop)
            i0, y0 = sp.localize_srp(st, frames)
            r_srp.append(sp.weighted_doa_error(st, i0, y0, s0, alpha))
            for k, b in enumerate(bases):
                i1, y1, _ = sp.localize(b, frames, "svd_exhaustive", "fp32")
                r_svd[k].append(sp.weighted_doa_error(st, i1, y1, s0, alpha))
        out[name] = {"K": [b.K for b in bases], "gain_Q_over_K": [2562 / b.K for b in bases],
                     "rmse_srp_mean": float(np.mean(r_srp)),
                     "rmse_svd_mean": [float(np.mean(r)) for r in r_svd],
                     "delta_rmse": [float(np.mean(r) - np.mean(r_srp)) for r in r_svd]}
    out["seconds"] = time.perf_counter() - t0
    return out


N_STREAMS, N_CONFIGS = 256, 16


def bench_batched(sp, I, torch, full=False):
    """The batched form: 256 streams in one CUDA-graph launch (autotuned, the GEMM1 kernel choice
    included).  Stream s uses one of 16 seeded configurations (array of 4-12 mics in a 5
    cm-radius ball, Q in {642, 2562}, N in {256, 512}; with full=True the whole range: 4-16
    mics, Q in {642, 2562, 10242}, N in {256, 512, 1024}; bases built once per configuration)
    and its own 50-2000 frames (a seeded slice of that configuration's 2000 frames).  Reported
    beside the same streams localised one sp_localize call after another, with the time to
    autotune the plan and to build it again from the tune cache (a file in a temporary
    directory)."""
    if full:
        cfgs = I.batched_streams(N_CONFIGS, M_range=(4, 16), Q_choices=(642, 2562, 10242),
                                 N_choices=(256, 512, 1024), T_range=(2000, 2000), seed_offset=200)
    else:
        cfgs = I.batched_streams(N_CONFIGS, M_range=(4, 12), Q_choices=(642, 2562), N_choices=(256, 512),
                                 T_range=(2000, 2000), seed_offset=100)
    bases, pools = [], []
    t0 = time.perf_counter()
    for wl in cfgs:
        st = sp.build_steering(wl["mic_xyz"], wl["dirs"], wl["fs"], wl["c"], wl["N"])
        bases.append(sp.svd_reduce(st, wl["delta"]))
        pools.append(torch.from_numpy(wl["frames"]).cuda())
    setup_s = time.perf_counter() - t0
    rng = np.random.default_rng(I.SEED_BASE + 2)
    sb, sf = [], []
    for s_ in range(N_STREAMS):
        c = int(rng.integers(0, N_CONFIGS))
        T = int(rng.integers(50, 2001))
        o = int(rng.integers(0, 2000 - T + 1))
        sb.append(bases[c])
        sf.append(pools[c][o:o + T].contiguous())
    total = sum(f.shape[0] for f in sf)
    with tempfile.TemporaryDirectory() as d:
        sp.set_tune_cache(os.path.join(d, "tune.json"))
        try:
            t0 = time.perf_counter()
            bt = sp.Batch(sb, sf, "svd_exhaustive", "fp16", autotune=True, tune_kernels=True)
            torch.cuda.synchronize()
            tune_s = time.perf_counter() - t0
            t0 = time.perf_counter()
            bt2 = sp.Batch(sb, sf, "svd_exhaustive", "fp16", autotune=True, tune_kernels=True)
            torch.cuda.synchronize()
            cached_s = time.perf_counter() - t0
            cached = bt2.info()["from_cache"]
            del bt2
        finally:
            sp.set_tune_cache(None)
    g_rate = _rate(bt.run, 10, total, torch)
    bt_g = sp.Batch(sb, sf, "svd_exhaustive", "fp16", group=True)   # the streams of a basis as one call
    grouped_rate = _rate(bt_g.run, 10, total, torch)
    grouped_info = bt_g.info()
    del bt_g

    def serial():   # FP32 where a basis has no tensor-core plan, as in the graph
        for b, f in zip(sb, sf):
            sp.localize(b, f, "svd_exhaustive", "fp32" if 2 * b.K > 288 else "fp16")
    s_rate = _rate(serial, 3, total, torch)
    ks = sorted({b.K for b in bases})
    ms = sorted({b.steering.M for b in bases})
    qs = sorted({b.steering.Q for b in bases})
    ns = sorted({b.steering.N for b in bases})
    return {"workload": f"{N_STREAMS} streams, {total} frames, {N_CONFIGS} configurations (M {ms[0]}-{ms[-1]}, "
                        f"Q {'/'.join(map(str, qs))}, N {'/'.join(map(str, ns))}, K {ks[0]}-{ks[-1]}), "
                        f"50-2000 frames per stream",
            "graph_frames_per_s": g_rate, "serial_frames_per_s": s_rate, "plan": bt.info(),
            "grouped_plan_frames_per_s": grouped_rate, "grouped_plan": grouped_info,
            "basis_setup_s": setup_s, "autotune_s": tune_s, "plan_from_cache_s": cached_s,
            "plan_from_cache": cached}


def _rate(fn, n, T, torch):
    fn()
    torch.cuda.synchronize()
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    a.record(stream)
    for _ in range(n):
        fn()
    z.record(stream)
    torch.cuda.synchronize()
    return T * n / (a.elapsed_time(z) / 1000)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp16", choices=["fp16", "bf16"])
    ap.add_argument("--frames", type=int, default=65536)
    ap.add_argument("--no-extras", action="store_true", help="skip the SRP / precision comparison lines")
    ap.add_argument("--only", choices=["array3d", "batched", "batched_default", "c5", "samples", "sweep", "kdtree"],
                    default=None,
                    help="run only one extra section and print its JSON (profiling runs)")
    ap.add_argument("--array3d-frames", type=int, default=C4_UNIQUE,
                    help="unique frames of the 3-D array section (repeated to 2^20 unless --only)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    __graft_entry__.build()
    import paper_1811_11785_gb300 as sp
    from paper_1811_11785_gb300 import inputs as I
    if args.only is not None:
        if args.only == "array3d":
            print(json.dumps(bench_array3d(sp, I, torch, args.array3d_frames, 1)), flush=True)
        elif args.only == "c5":
            print(json.dumps(bench_c5(sp, I, torch)), flush=True)
        elif args.only == "samples":
            print(json.dumps(bench_samples(sp, I, torch)), flush=True)
        elif args.only == "sweep":
            print(json.dumps(bench_delta_sweep(sp, I, torch)), flush=True)
        elif args.only == "kdtree":
            print(json.dumps(bench_kdtree(sp, I, torch)), flush=True)
        elif args.only == "batched_default":
            print(json.dumps(bench_batched(sp, I, torch)), flush=True)
        else:
            print(json.dumps(bench_batched(sp, I, torch, full=True)), flush=True)
        return

    def lib_project(b, frames, prec, zout):
        rc = sp.lib().sp_project(b.handle, ctypes.c_void_p(frames.data_ptr()), frames.shape[0], sp.PREC[prec],
                                 ctypes.c_void_p(zout.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0, sp.lib().sp_last_error()

    T = args.frames
    wl = I.workload(WORKLOAD, T=T, seed_offset=rank)
    st = sp.build_steering(wl["mic_xyz"], wl["dirs"], wl["fs"], wl["c"], wl["N"], materialize_w=True)
    b = sp.svd_reduce(st, wl["delta"])
    frames = torch.from_numpy(wl["frames"]).cuda()
    frames_host = torch.from_numpy(wl["frames"]).pin_memory()
    idx = torch.empty(T, dtype=torch.int32, device="cuda")
    score = torch.empty(T, dtype=torch.float32, device="cuda")
    proj = torch.empty(T, dtype=torch.float32, device="cuda")
    out = (idx, score, proj)
    stream = torch.cuda.current_stream()

    def step():
        sp.localize(b, frames, "svd_exhaustive", args.prec, out=out)

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    sp.check_status()

    clocks = Clocks(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    sp.check_status()

    # per-kernel durations on the launching stream: the dominant kernel (fused PHAT + GEMM1,
    # svd_proj_tma_kernel) alone through sp_project, then + the scan, then + online step 4
    zbuf = torch.empty((T, b.K), dtype=torch.complex64, device="cuda")
    kout = (idx, None, proj)

    def avg_ms(fn, n):
        for _ in range(3):
            fn()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n):
            fn()
        z.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(z) / n

    k_ms = avg_ms(lambda: lib_project(b, frames, args.prec, zbuf), args.steps)
    scan_ms = avg_ms(lambda: sp.localize(b, frames, "svd_exhaustive", args.prec, out=kout), args.steps) - k_ms
    step4_ms = ms / args.steps - k_ms - scan_ms

    # end to end through the host-buffer entry point: H2D of the frames and D2H of the results
    hout = (torch.empty(T, dtype=torch.int32).pin_memory(), torch.empty(T, dtype=torch.float32).pin_memory(),
            torch.empty(T, dtype=torch.float32).pin_memory())
    sp.localize_host(b, frames_host, "svd_exhaustive", args.prec, out=hout)
    barrier()
    e2e_steps = max(3, args.steps // 2)
    e2e_times = []
    for _ in range(e2e_steps):   # each step timed on its own; the median (the host link is shared)
        t0 = time.perf_counter()
        sp.localize_host(b, frames_host, "svd_exhaustive", args.prec, out=hout)
        barrier()
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = statistics.median(e2e_times)
    # the host link alone: one plain pinned host -> device copy of the same frames
    dst = torch.empty_like(frames)
    dst.copy_(frames_host, non_blocking=True)
    barrier()
    t0 = time.perf_counter()
    for _ in range(3):
        dst.copy_(frames_host, non_blocking=True)
    barrier()
    h2d_gbs = 3 * frames_host.numel() * 8 / (time.perf_counter() - t0) / 1e9
    del dst

    # max over ranks
    if ws > 1:
        tt = torch.tensor([ms, e2e_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms, e2e_s = float(tt[0]), float(tt[1])

    extras = {}
    if rank == 0:
        # agreement with the FP64 oracle on a sample + the oracle's own CPU throughput
        rate, dt, sel, ref, Y, cls = oracle_sample(wl, 2048)
        gi = idx.cpu().numpy()[sel]
        agree = float(np.mean(cls[gi] == cls[ref]))
        # score errors against the FP64 oracle on the same sample, in units of L (|Y| <= L)
        import oracle as O
        last = oracle_sample.last
        Lr = float(last["L"])
        proj_err = float(np.max(np.abs(proj.cpu().numpy()[sel] - Y[np.arange(len(sel)), gi]))) / Lr
        s4_err = float(np.max(np.abs(score.cpu().numpy()[sel] - oracle_step4(gi, wl["N"])))) / Lr
        if not args.no_extras:
            # plain FP32 SRP-PHAT (the reference form) and the other precisions, same frames
            def rate_of(fn, n):
                fn()
                torch.cuda.synchronize()
                a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(n):
                    fn()
                z.record(stream)
                torch.cuda.synchronize()
                return T * n / (a.elapsed_time(z) / 1000)
            extras["srp_fp32_frames_per_s"] = rate_of(lambda: sp.localize_srp(st, frames), 2)
            # plain SRP-PHAT is FP32-ALU bound: 4 Q L flops per frame (Eq. 9) against the FP32 FMA
            # rate measured on this GPU by the library's own microbenchmark (sp_fp32_fma_peak)
            alu_peak = sp.fp32_fma_peak()
            sm_count = torch.cuda.get_device_properties(0).multi_processor_count
            srp_tflops = extras["srp_fp32_frames_per_s"] * 4.0 * st.Q * st.L / 1e12
            extras["srp_fp32_roofline"] = {"bound": "alu", "achieved": srp_tflops, "peak": alu_peak,
                                           "unit": "TFLOP/s", "frac": srp_tflops / alu_peak,
                                           "peak_source": "measured: sp_fp32_fma_peak (independent FMA chains "
                                                          f"on all {sm_count} SMs, CUDA events)"}
            extras["svd_fp32_frames_per_s"] = rate_of(lambda: sp.localize(b, frames, "svd_exhaustive", "fp32"), 3)
            other = "bf16" if args.prec == "fp16" else "fp16"
            extras[f"svd_{other}_frames_per_s"] = rate_of(lambda: sp.localize(b, frames, "svd_exhaustive", other), 5)
            extras["svd_kdtree_fp16_frames_per_s"] = rate_of(lambda: sp.localize(b, frames, "svd_kdtree", "fp16"), 3)
            extras["kdtree_search"] = kdtree_stats(sp, b, frames, torch)
            extras["from_samples"] = bench_samples(sp, I, torch)
            extras["delta_sweep"] = bench_delta_sweep(sp, I, torch)
            extras["array3d_q10242"] = bench_array3d(sp, I, torch, args.array3d_frames, C4_REPEAT)
            extras["batched_256_streams"] = bench_batched(sp, I, torch)

        peak, peak_kind = _peaks()
        frame_bytes = st.M * st.B * 8                       # the STFT of one frame
        per_frame_bytes = frame_bytes                       # algorithmic bytes of the dominant kernel
        achieved = per_frame_bytes * T / (k_ms / 1000) / 1e9
        line = {
            "metric": METRIC, "value": T * ws * args.steps / (ms / 1000), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.prec,
            "data": "synthetic",
            "config": arm_config(b.K, T),
            "agreement_vs_oracle": agree, "agreement_sample_frames": int(len(sel)),
            "score_error_vs_oracle": {"search_score_max_over_L": proj_err, "step4_score_max_over_L": s4_err},
            "gpu_launches": 5 * args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": TRAFFIC_PER_FRAME and TRAFFIC_PER_FRAME * T,
                         "kernel": DOMINANT_KERNEL, "kernel_ms": k_ms, "peak_source": peak_kind,
                         "algorithmic_bytes_per_frame": per_frame_bytes},
            "kernel_ms": {DOMINANT_KERNEL: k_ms, "svd_scan_kernel": scan_ms, "step4_bulk_kernel": step4_ms},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": _cores(), "kind": "oracle",
                             "sample": f"2048 frames of the same workload (PHAT, Z = V^H X, Re{{D Z}} argmax, "
                                       f"online step 4 in FP64 numpy), split over {_cores()} spawned processes "
                                       "with one BLAS thread each"},
            "e2e": {"value": T * ws / e2e_s, "unit": UNIT, "h2d_bytes_per_step": T * frame_bytes,
                    "d2h_bytes_per_step": T * 12, "host_to_device_copy_GBps": h2d_gbs,
                    "timing": f"median of {e2e_steps} steps, each timed alone (max over ranks)"},
            "clocks": clk,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
