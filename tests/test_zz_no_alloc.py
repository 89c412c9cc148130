"""sp_localize_noalloc: the localisation entry point for callers that cannot allocate
device memory on their processing path (real-time audio callbacks, plugin hosts, fixed
memory budgets).  It keeps its scratch in a fixed array inside the library, so it must
give the same results as sp_localize, call after call, while the array holds whatever
the previous call left in it.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import paper_1811_11785_gb300 as sp
from paper_1811_11785_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import __graft_entry__
    __graft_entry__.build()
    wl = I.workload("planar_q2562", T=3000)
    st = sp.build_steering(wl["mic_xyz"], wl["dirs"], wl["fs"], wl["c"], wl["N"])
    b = sp.svd_reduce(st, wl["delta"])
    frames = torch.from_numpy(wl["frames"]).cuda()
    return st, b, frames


def _noalloc_via_c_abi(b, frames, prec):
    T = frames.shape[0]
    idx = torch.full((T,), -7, dtype=torch.int32, device="cuda")
    score = torch.full((T,), float("nan"), dtype=torch.float32, device="cuda")
    proj = torch.full((T,), float("nan"), dtype=torch.float32, device="cuda")
    rc = sp.lib().sp_localize_noalloc(b.handle, ctypes.c_void_p(frames.data_ptr()), T, sp.PREC[prec],
                                      ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(score.data_ptr()),
                                      ctypes.c_void_p(proj.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, sp.lib().sp_last_error().decode()
    return idx, score, proj


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_noalloc_matches_localize_two_calls_in_a_row(setup, prec):
    st, b, frames = setup
    L = st.L
    # two calls in a row on different frames: the second sees the first call's leftovers
    for lo, hi in [(0, 3000), (517, 1290)]:
        fr = frames[lo:hi].contiguous()
        i1, s1, p1 = sp.localize(b, fr, "svd_exhaustive", prec)
        i2, s2, p2 = _noalloc_via_c_abi(b, fr, prec)
        torch.cuda.synchronize()
        sp.check_status()
        assert torch.equal(i1, i2)
        assert np.max(np.abs(p1.cpu().numpy() - p2.cpu().numpy())) <= 1e-5 * L
        assert np.max(np.abs(s1.cpu().numpy() - s2.cpu().numpy())) <= 1e-5 * L


SCRATCH_BYTES = 8 << 20


def _scratch_need(T, K):
    """Bytes of the built-in array a call of T frames uses: Z (T x K complex64), ||Z||^2
    (T floats) and the scan's overflow list (a count, T indices, T keys), each region rounded
    up to 256 bytes."""
    r = lambda n: (n + 255) // 256 * 256
    return r(T * K * 8) + r(T * 4) + 256 + r(T * 4) + T * 8


def _largest_T(K):
    T = SCRATCH_BYTES // (8 * K + 16)
    while _scratch_need(T + 1, K) <= SCRATCH_BYTES:
        T += 1
    while _scratch_need(T, K) > SCRATCH_BYTES:
        T -= 1
    return T


def test_noalloc_warm_up_call_launches_nothing(setup):
    """T == 0 is the warm-up call (scratch address, kernel loading): it succeeds without frames
    or outputs, and the next call still matches sp_localize."""
    st, b, frames = setup
    rc = sp.lib().sp_localize_noalloc(b.handle, None, 0, sp.PREC["fp16"], None, None, None, None)
    assert rc == 0, sp.lib().sp_last_error().decode()
    i1, _, p1 = sp.localize(b, frames[:300].contiguous(), "svd_exhaustive", "fp16")
    i2, _, p2 = _noalloc_via_c_abi(b, frames[:300].contiguous(), "fp16")
    torch.cuda.synchronize()
    assert torch.equal(i1, i2) and torch.equal(p1, p2)


def test_noalloc_at_its_largest_batch(setup):
    """The largest T whose scratch fits the 8 MiB array (its last region ends at the array's
    end) matches sp_localize; one frame more is rejected before any work."""
    st, b, frames = setup
    Tmax = _largest_T(b.K)
    assert _scratch_need(Tmax, b.K) <= SCRATCH_BYTES < _scratch_need(Tmax + 1, b.K)
    reps = (Tmax + frames.shape[0]) // frames.shape[0]
    fr = frames.repeat(reps, 1, 1)[:Tmax + 1].contiguous()
    i1, s1, p1 = sp.localize(b, fr[:Tmax], "svd_exhaustive", "fp16")
    i2, s2, p2 = _noalloc_via_c_abi(b, fr[:Tmax], "fp16")
    torch.cuda.synchronize()
    sp.check_status()
    assert torch.equal(i1, i2)
    assert np.max(np.abs(p1.cpu().numpy() - p2.cpu().numpy())) <= 1e-5 * st.L
    assert np.max(np.abs(s1.cpu().numpy() - s2.cpu().numpy())) <= 1e-5 * st.L
    idx = torch.empty(Tmax + 1, dtype=torch.int32, device="cuda")
    rc = sp.lib().sp_localize_noalloc(b.handle, ctypes.c_void_p(fr.data_ptr()), Tmax + 1, sp.PREC["fp16"],
                                      ctypes.c_void_p(idx.data_ptr()), None, None, None)
    assert rc == sp.api.SP_EINVAL
    assert b"exceeds" in sp.lib().sp_last_error()


def test_noalloc_python_wrapper_optional_outputs(setup):
    """The Python binding with the score and projection outputs left out gives the same
    indices as sp_localize."""
    st, b, frames = setup
    fr = frames[100:900].contiguous()
    idx, sc, pj = sp.localize_noalloc(b, fr, "bf16", score=False, proj=False)
    assert sc is None and pj is None
    ref = sp.localize(b, fr, "svd_exhaustive", "bf16", score=False, proj=False)[0]
    torch.cuda.synchronize()
    assert torch.equal(idx, ref)


def test_noalloc_checks_arguments_like_localize(setup):
    st, b, frames = setup
    T = 64
    idx = torch.empty(T, dtype=torch.int32, device="cuda")
    score = torch.empty(T + 1, dtype=torch.float32, device="cuda")
    f = ctypes.c_void_p(frames.data_ptr())
    lib = sp.lib()
    # a misaligned score or projection pointer, and T beyond 2^28, are SP_EINVAL as in sp_localize
    bad = ctypes.c_void_p(score.data_ptr() + 2)
    assert lib.sp_localize_noalloc(b.handle, f, T, sp.PREC["fp16"], ctypes.c_void_p(idx.data_ptr()), bad, None,
                                   None) == sp.api.SP_EINVAL
    assert lib.sp_localize_noalloc(b.handle, f, T, sp.PREC["fp16"], ctypes.c_void_p(idx.data_ptr()), None, bad,
                                   None) == sp.api.SP_EINVAL
    assert lib.sp_localize_noalloc(b.handle, f, (1 << 28) + 1, sp.PREC["fp16"], ctypes.c_void_p(idx.data_ptr()),
                                   None, None, None) == sp.api.SP_EINVAL
    assert lib.sp_localize_noalloc(b.handle, f, T, sp.PREC["fp32"], ctypes.c_void_p(idx.data_ptr()), None, None,
                                   None) == sp.api.SP_ENOTIMPL
