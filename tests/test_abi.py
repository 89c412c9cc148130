"""The C ABI builds and loads on the host, exports every entry point include/svdphat.h
declares, and rejects bad arguments before touching the GPU (no compute calls here)."""
import ctypes
import os
import re

import numpy as np
import pytest

import __graft_entry__
import paper_1811_11785_gb300 as sp
from paper_1811_11785_gb300 import api

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "svdphat.h")


def header_functions():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sp_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return sp.lib()


def test_header_declares_the_boundary():
    names = header_functions()
    for must in ["sp_build_steering", "sp_svd_reduce", "sp_localize", "sp_phat", "sp_project",
                 "sp_localize_srp", "sp_localize_host", "sp_last_error", "sp_check_status"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name
    assert set(header_functions()) == set(api.exported_symbols())


def test_version_and_error_string(lib):
    assert lib.sp_version() >= 100
    assert isinstance(lib.sp_last_error(), bytes)


def _bs(lib, M=3, Q=4, N=16, fs=16000.0, c=343.0, flags=0, null_out=False, zero_dir=False, nan_dir=False,
        near=False):
    mic = np.zeros((M, 3))
    mic[:, 0] = np.arange(M) * 0.01
    d = np.tile([0.0, 0.0, 1.0], (max(Q, 1), 1))
    if zero_dir:
        d[0] = 0.0
    if nan_dir:
        d[0, 1] = np.nan
    h = ctypes.c_void_p()
    dp = ctypes.POINTER(ctypes.c_double)
    fn = lib.sp_build_steering_nearfield if near else lib.sp_build_steering
    return fn(mic.ctypes.data_as(dp), M, d.ctypes.data_as(dp), Q, fs, c, N, flags,
              None if null_out else ctypes.byref(h))


BAD_STEERING = [dict(M=1), dict(M=65), dict(Q=0), dict(N=15), dict(N=2), dict(fs=0.0), dict(c=-1.0), dict(flags=8),
                dict(null_out=True), dict(zero_dir=True), dict(nan_dir=True)]


@pytest.mark.parametrize("near", [False, True])
@pytest.mark.parametrize("kw", BAD_STEERING)
def test_build_steering_rejects_bad_arguments(lib, kw, near):
    """Both builders (directions, Eq. 2; source positions, Eq. 1) refuse bad geometry with
    SP_EINVAL on the host, naming themselves in the message."""
    assert _bs(lib, near=near, **kw) == api.SP_EINVAL
    msg = lib.sp_last_error()
    assert msg.startswith(b"sp_build_steering_nearfield" if near else b"sp_build_steering:")
    if kw.get("zero_dir"):
        assert (b"origin" in msg) if near else (b"zero direction" in msg)


def test_steering_model_query_rejects_null(lib):
    nf = ctypes.c_int()
    assert lib.sp_steering_nearfield(None, ctypes.byref(nf)) == api.SP_EINVAL


def test_other_entry_points_reject_null_handles(lib):
    assert lib.sp_svd_reduce(None, 1e-5, 0, None, None) == api.SP_EINVAL
    out = ctypes.c_void_p()
    assert lib.sp_svd_reduce(None, 1e-5, 0, ctypes.byref(out), None) == api.SP_EINVAL
    assert lib.sp_localize(None, None, 4, 1, 1, None, None, None, None) == api.SP_EINVAL
    assert lib.sp_localize_srp(None, None, 4, None, None, None) == api.SP_EINVAL
    assert lib.sp_project(None, None, 4, 1, None, None) == api.SP_EINVAL
    assert lib.sp_phat(None, -1, 3, 5, None, None) == api.SP_EINVAL
    assert lib.sp_phat(None, 0, 3, 5, None, None) == api.SP_OK  # T = 0 is a no-op
    assert lib.sp_phat(None, 2, 1, 5, None, None) == api.SP_EINVAL
    assert lib.sp_basis_info(None, None, None, None, 0) == api.SP_EINVAL
    lib.sp_steering_destroy(None)
    lib.sp_basis_destroy(None)


def _basis_file(path, M=3, Q=4, N=16, K=2, n_sigma=3, magic=b"SVDPHAT1", version=1, corrupt=0, truncate=0):
    """A file in the documented basis layout (header, FP64 payload, FNV-1a 64 checksum)."""
    import struct
    P, B = M * (M - 1) // 2, N // 2 + 1
    L = P * B
    nd = 3 * M + 3 * Q + n_sigma + 2 * L * K + 2 * Q * K
    hdr = magic + struct.pack("<II6i3dQQ", version, 80, M, Q, N, K, n_sigma, 0, 16000.0, 343.0, 1e-5, nd * 8, 0)
    body = np.ones(nd).tobytes()
    h = 1469598103934665603
    for byte in hdr + body:
        h = ((h ^ byte) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    data = bytearray(hdr + body + struct.pack("<Q", h))
    if corrupt:
        data[80 + corrupt] ^= 0x40
    if truncate:
        data = data[:-truncate]
    with open(path, "wb") as f:
        f.write(bytes(data))


@pytest.mark.parametrize("kw", [dict(magic=b"SVDPHAT0"), dict(version=2), dict(corrupt=17), dict(truncate=8),
                                dict(K=0), dict(K=5), dict(n_sigma=1), dict(N=15), dict(M=1)])
def test_load_basis_rejects_malformed_files(lib, tmp_path, kw):
    """Every malformed file is refused with SP_EINVAL before any device work."""
    path = str(tmp_path / "basis.bin")
    _basis_file(path, **kw)
    out = ctypes.c_void_p(1)
    assert lib.sp_load_basis(path.encode(), 0, ctypes.byref(out), None) == api.SP_EINVAL
    assert out.value is None
    assert len(lib.sp_last_error()) > 0


def test_load_basis_rejects_missing_file_and_null_arguments(lib, tmp_path):
    out = ctypes.c_void_p()
    assert lib.sp_load_basis(str(tmp_path / "none.bin").encode(), 0, ctypes.byref(out), None) == api.SP_EINVAL
    assert lib.sp_load_basis(None, 0, ctypes.byref(out), None) == api.SP_EINVAL
    assert lib.sp_load_basis(b"x", 0, None, None) == api.SP_EINVAL
    assert lib.sp_load_basis(b"x", 4, ctypes.byref(out), None) == api.SP_EINVAL
    assert lib.sp_save_basis(None, b"x") == api.SP_EINVAL
    assert lib.sp_basis_steering(None, ctypes.byref(out)) == api.SP_EINVAL


def test_batch_and_proposal_calls_reject_bad_arguments(lib):
    out = ctypes.c_void_p()
    assert lib.sp_batch_create(0, None, None, None, 1, 1, None, None, None, 0, None, ctypes.byref(out)) == api.SP_EINVAL
    assert lib.sp_batch_create(1, None, None, None, 1, 1, None, None, None, 0, None, None) == api.SP_EINVAL
    assert lib.sp_batch_create(1, None, None, None, 1, 1, None, None, None, 0, None, ctypes.byref(out)) == api.SP_EINVAL
    assert lib.sp_batch_run(None, None) == api.SP_EINVAL
    assert lib.sp_batch_info(None, None, None, None, None, None, None, None, None) == api.SP_EINVAL
    lib.sp_batch_destroy(None)
    assert lib.sp_proposal_create(None, None, 642, 256, 256, 0, ctypes.byref(out)) == api.SP_EINVAL
    assert lib.sp_proposal_create(None, None, 642, 256, 256, 0, None) == api.SP_EINVAL
    assert lib.sp_localize_learned(None, None, 4, 1, 4, ctypes.c_float(0.5), None, None, None, None, None) == api.SP_EINVAL
    assert lib.sp_proposal_dims(None, None, None, None, None, None) == api.SP_EINVAL
    assert lib.sp_proposal_train_step(None, None, None, None, 4, ctypes.c_float(1e-3), None, None) == api.SP_EINVAL
    lib.sp_proposal_destroy(None)


def test_debug_build_compiles_and_exports_every_symbol():
    """The SP_DEBUG build (device bounds checks) compiles for sm_103a and exports the same ABI."""
    from paper_1811_11785_gb300 import build as B
    path = B.build(debug=True)
    L = ctypes.CDLL(path)
    for name in header_functions():
        assert hasattr(L, name), name
