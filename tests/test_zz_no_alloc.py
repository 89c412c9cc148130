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


def test_noalloc_rejects_batches_beyond_its_scratch(setup):
    st, b, frames = setup
    big = 8 * 2 ** 20 // (8 * b.K + 16) + 1   # more frames than the built-in array holds
    idx = torch.empty(1, dtype=torch.int32, device="cuda")
    rc = sp.lib().sp_localize_noalloc(b.handle, ctypes.c_void_p(frames.data_ptr()), big, sp.PREC["fp16"],
                                      ctypes.c_void_p(idx.data_ptr()), None, None, None)
    assert rc == sp.api.SP_EINVAL
    assert b"exceeds" in sp.lib().sp_last_error()
