"""The SP_DEBUG build (libsvdphat_debug.so: device bounds checks that record a failure in the
status word, sp_check_status -> SP_EBOUNDS) runs the main paths without a failed check and gives
the release build's results.  It runs in a child process that loads the debug library."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import paper_1811_11785_gb300 as sp
from paper_1811_11785_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
import paper_1811_11785_gb300 as sp
from paper_1811_11785_gb300 import inputs as I
assert sp.lib()._name.endswith("libsvdphat_debug.so"), sp.lib()._name
wl = I.workload("planar_q2562", T=700)
st = sp.build_steering(wl["mic_xyz"], wl["dirs"], wl["fs"], wl["c"], wl["N"], materialize_w=True)
b = sp.svd_reduce(st, wl["delta"])
fr = torch.from_numpy(wl["frames"]).cuda()
out = {}
for mode, prec in [("svd_exhaustive", "fp16"), ("svd_exhaustive", "bf16"), ("svd_exhaustive", "fp32"),
                   ("svd_kdtree", "fp16")]:
    out[mode + "_" + prec] = sp.localize(b, fr, mode, prec)[0].cpu().numpy()
out["srp"] = sp.localize_srp(st, fr)[0].cpu().numpy()
x = torch.from_numpy(I.time_signals(np.random.default_rng(3), wl["mic_xyz"], 40000, 16000.0, 343.0,
                                    np.array([0.0, 0.6, 0.8]), 10.0)).cuda()
out["samples"] = sp.localize_samples(b, x, 256)[0].cpu().numpy()
torch.cuda.synchronize()
sp.check_status()
np.savez(sys.argv[2], **out)
print("debug build ok")
'''


def test_debug_build_runs_clean_and_matches_release(tmp_path):
    import __graft_entry__
    __graft_entry__.build()
    from paper_1811_11785_gb300 import build as B
    dbg = B.build(debug=True)
    script = tmp_path / "child.py"
    script.write_text(CHILD)
    res = tmp_path / "debug.npz"
    env = dict(os.environ, SVDPHAT_LIB=dbg)
    r = subprocess.run([sys.executable, str(script), ROOT, str(res)], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    got = np.load(res)
    wl = I.workload("planar_q2562", T=700)
    st = sp.build_steering(wl["mic_xyz"], wl["dirs"], wl["fs"], wl["c"], wl["N"], materialize_w=True)
    b = sp.svd_reduce(st, wl["delta"])
    fr = torch.from_numpy(wl["frames"]).cuda()
    for mode, prec in [("svd_exhaustive", "fp16"), ("svd_exhaustive", "bf16"), ("svd_exhaustive", "fp32"),
                       ("svd_kdtree", "fp16")]:
        assert np.array_equal(got[mode + "_" + prec], sp.localize(b, fr, mode, prec)[0].cpu().numpy()), mode + prec
    assert np.array_equal(got["srp"], sp.localize_srp(st, fr)[0].cpu().numpy())
