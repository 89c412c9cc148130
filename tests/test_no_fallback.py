"""The product path has no CPU fallback: without its CUDA library, or without a GPU, a call
fails loudly, and the package never imports the oracle."""
import os
import subprocess
import sys

import pytest
import torch

import paper_1811_11785_gb300 as sp
from paper_1811_11785_gb300 import api
from paper_1811_11785_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_package_never_imports_the_oracle():
    code = ("import sys; sys.path.insert(0, %r); import paper_1811_11785_gb300, paper_1811_11785_gb300.api; "
            "assert 'oracle' not in sys.modules and not any(m.startswith('oracle.') for m in sys.modules)" % ROOT)
    subprocess.run([sys.executable, "-c", code], check=True, cwd=ROOT)


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(api, "_lib", None)
    monkeypatch.setattr(api._build, "LIB", str(tmp_path / "libsvdphat.so"))
    with pytest.raises(RuntimeError, match="not built"):
        api.lib()


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour on a host without a GPU")
def test_calls_without_a_gpu_raise():
    import __graft_entry__
    __graft_entry__.build()
    with pytest.raises(sp.SvdPhatError):
        sp.build_steering(I.array_3d(), I.icosphere(1), 16000.0, 343.0, 64)
    with pytest.raises(sp.SvdPhatError):
        sp.build_steering_nearfield(I.array_3d(), I.nearfield_points(1, radii=(0.5,)), 16000.0, 343.0, 64)
