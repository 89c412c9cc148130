"""Thin Python binding of libsvdphat.so (``include/svdphat.h``): argument marshalling only.

Every step of the localisation path runs in the library's CUDA kernels; PyTorch only
provides device memory and the current CUDA stream.  There is no fallback: if the shared
library has not been built (``paper_1811_11785_gb300.build.build()``) or there is no GPU,
calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

MODE = {"srp": 0, "svd_exhaustive": 1, "svd_kdtree": 2, "svd_learned": 3}
PREC = {"fp32": 0, "fp16": 1, "bf16": 2}
STEER_MATERIALIZE_W = 1

SP_OK, SP_EINVAL, SP_ENOMEM, SP_ECUDA, SP_ETIMEOUT, SP_ENOTIMPL = 0, -1, -2, -3, -4, -5


class SvdPhatError(RuntimeError):
    def __init__(self, fn: str, code: int, msg: str):
        super().__init__(f"{fn} failed with code {code}: {msg}")
        self.code = code


_lib = None

_vp = ctypes.c_void_p
_ip = ctypes.POINTER(ctypes.c_int)
_dp = ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "sp_last_error": ([], ctypes.c_char_p),
    "sp_version": ([], ctypes.c_int),
    "sp_build_steering": ([_dp, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                           ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)], ctypes.c_int),
    "sp_build_steering_nearfield": ([_dp, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)], ctypes.c_int),
    "sp_steering_nearfield": ([_vp, _ip], ctypes.c_int),
    "sp_steering_dims": ([_vp, _ip, _ip, _ip, _ip, _ip], ctypes.c_int),
    "sp_steering_classes": ([_vp, _ip, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "sp_steering_tau": ([_vp, _dp], ctypes.c_int),
    "sp_steering_w": ([_vp, _vp, _vp], ctypes.c_int),
    "sp_steering_destroy": ([_vp], None),
    "sp_svd_reduce": ([_vp, ctypes.c_double, ctypes.c_int, ctypes.POINTER(_vp), _ip], ctypes.c_int),
    "sp_basis_info": ([_vp, _ip, _ip, _dp, ctypes.c_int], ctypes.c_int),
    "sp_basis_v": ([_vp, _dp], ctypes.c_int),
    "sp_basis_d": ([_vp, _dp], ctypes.c_int),
    "sp_basis_kdtree_info": ([_vp, _ip, _ip, _ip], ctypes.c_int),
    "sp_basis_destroy": ([_vp], None),
    "sp_save_basis": ([_vp, ctypes.c_char_p], ctypes.c_int),
    "sp_load_basis": ([ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(_vp), _ip], ctypes.c_int),
    "sp_basis_steering": ([_vp, ctypes.POINTER(_vp)], ctypes.c_int),
    "sp_phat": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp], ctypes.c_int),
    "sp_project": ([_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp], ctypes.c_int),
    "sp_localize": ([_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp], ctypes.c_int),
    "sp_localize_srp": ([_vp, _vp, ctypes.c_int, _vp, _vp, _vp], ctypes.c_int),
    "sp_localize_host": ([_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int,
                          _vp], ctypes.c_int),
    "sp_localize_noalloc": ([_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp], ctypes.c_int),
    "sp_check_status": ([_vp], ctypes.c_int),
    "sp_proposal_create": ([_vp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong,
                            ctypes.POINTER(_vp)], ctypes.c_int),
    "sp_proposal_destroy": ([_vp], None),
    "sp_proposal_dims": ([_vp, _ip, _ip, _ip, _ip, ctypes.POINTER(ctypes.c_longlong)], ctypes.c_int),
    "sp_proposal_cells": ([_vp, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "sp_proposal_get_params": ([_vp, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
    "sp_proposal_set_params": ([_vp, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
    "sp_proposal_examples": ([_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp], ctypes.c_int),
    "sp_proposal_forward_f32": ([_vp, _vp, ctypes.c_int, _vp, _vp], ctypes.c_int),
    "sp_proposal_grad": ([_vp, _vp, _vp, ctypes.c_int, _vp, _vp, _vp], ctypes.c_int),
    "sp_proposal_train_step": ([_vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_float, _vp, _vp], ctypes.c_int),
    "sp_proposal_infer": ([_vp, _vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp], ctypes.c_int),
    "sp_batch_create": ([ctypes.c_int, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int, _vp,
                         ctypes.POINTER(_vp)], ctypes.c_int),
    "sp_batch_run": ([_vp, _vp], ctypes.c_int),
    "sp_batch_info": ([_vp, _ip, _ip, _ip, ctypes.POINTER(ctypes.c_float), _ip, _ip, _ip, _ip], ctypes.c_int),
    "sp_set_tune_cache": ([ctypes.c_char_p], ctypes.c_int),
    "sp_tune_cache_get": ([ctypes.c_char_p, _ip, _ip, _ip, ctypes.POINTER(ctypes.c_float), _ip, _ip], ctypes.c_int),
    "sp_tune_cache_put": ([ctypes.c_char_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_int],
                          ctypes.c_int),
    "sp_batch_destroy": ([_vp], None),
    "sp_localize_batched": ([ctypes.c_int, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp],
                            ctypes.c_int),
    "sp_localize_learned": ([_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float, _vp, _vp, _vp, _vp,
                             _vp], ctypes.c_int),
    "sp_set_wait_budget": ([ctypes.c_longlong], ctypes.c_int),
    "sp_fp32_fma_peak": ([ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "sp_kdtree_search": ([_vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp], ctypes.c_int),
    "sp_stft": ([_vp, ctypes.c_int, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, _vp, _vp,
                 ctypes.POINTER(ctypes.c_int), _vp], ctypes.c_int),
    "sp_apply_mask": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp], ctypes.c_int),
    "sp_weighted_doa_error": ([_vp, _vp, _vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                               _vp], ctypes.c_int),
    "sp_localize_samples": ([_vp, _vp, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_int, _vp, ctypes.c_int,
                             ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp], ctypes.c_int),
}


def exported_symbols() -> list[str]:
    return list(_SIGS)


def lib():
    """Load libsvdphat.so (built in-tree; SVDPHAT_LIB may name another build of it, e.g. the
    SP_DEBUG build libsvdphat_debug.so); raise if it is missing."""
    global _lib
    if _lib is None:
        path = os.environ.get("SVDPHAT_LIB") or _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is not built; call paper_1811_11785_gb300.build.build() first")
        L = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(fn: str, rc: int):
    if rc != SP_OK:
        raise SvdPhatError(fn, rc, lib().sp_last_error().decode())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _mode(m):
    return MODE[m] if isinstance(m, str) else int(m)


def _prec(p):
    return PREC[p] if isinstance(p, str) else int(p)


def _frames(frames, st):
    import torch
    if not (isinstance(frames, torch.Tensor) and frames.is_cuda and frames.dtype == torch.complex64):
        raise TypeError("frames must be a CUDA complex64 tensor [T][M][N/2+1]")
    if not frames.is_contiguous():
        raise ValueError("frames must be contiguous")
    if frames.dim() != 3 or (st is not None and (frames.shape[1] != st.M or frames.shape[2] != st.B)):
        raise ValueError("frames must have shape [T][M][N/2+1] matching the steering handle")
    return frames


class Steering:
    """TDOA table and steering matrix W (Eq. 2, 4, 8) on the device; with nearfield=True
    ``dirs`` are source positions and the TDOA follows Eq. 1."""

    def __init__(self, mic_xyz, dirs, fs: float, c: float, N: int, materialize_w: bool = False,
                 nearfield: bool = False):
        L = lib()
        mic = np.ascontiguousarray(mic_xyz, dtype=np.float64)
        d = np.ascontiguousarray(dirs, dtype=np.float64)
        h = _vp()
        fn = "sp_build_steering_nearfield" if nearfield else "sp_build_steering"
        _check(fn, getattr(L, fn)(mic.ctypes.data_as(_dp), mic.shape[0], d.ctypes.data_as(_dp), d.shape[0],
                                  float(fs), float(c), int(N), STEER_MATERIALIZE_W if materialize_w else 0,
                                  ctypes.byref(h)))
        self._h = h
        self._owned = True
        self._dims()
        self.materialized = materialize_w

    @classmethod
    def _borrowed(cls, h, materialized: bool):
        """A view of a steering handle owned by a loaded basis (never destroyed here)."""
        self = cls.__new__(cls)
        self._h = h
        self._owned = False
        self._dims()
        self.materialized = materialized
        return self

    def _dims(self):
        v = [ctypes.c_int() for _ in range(5)]
        _check("sp_steering_dims", lib().sp_steering_dims(self._h, *[ctypes.byref(x) for x in v]))
        self.M, self.P, self.Q, self.N, self.B = (x.value for x in v)
        self.L = self.P * self.B
        nf = ctypes.c_int()
        _check("sp_steering_nearfield", lib().sp_steering_nearfield(self._h, ctypes.byref(nf)))
        self.nearfield = bool(nf.value)

    @property
    def handle(self):
        return self._h

    def classes(self) -> np.ndarray:
        """For every direction, the lowest index of its class (identical TDOA vectors)."""
        out = np.empty(self.Q, dtype=np.int32)
        _check("sp_steering_classes", lib().sp_steering_classes(
            self._h, None, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
        return out

    def tau(self) -> np.ndarray:
        out = np.empty((self.Q, self.P), dtype=np.float64)
        _check("sp_steering_tau", lib().sp_steering_tau(self._h, out.ctypes.data_as(_dp)))
        return out

    def w(self):
        import torch
        out = torch.empty((self.Q, self.L), dtype=torch.complex64, device="cuda")
        _check("sp_steering_w", lib().sp_steering_w(self._h, _ptr(out), _stream()))
        return out

    def __del__(self):
        h = getattr(self, "_h", None)
        if getattr(self, "_owned", False) and h is not None and h.value and _lib is not None:
            _lib.sp_steering_destroy(h)
            self._h = None


class Basis:
    """Rank-K basis (V, D = U S, D^) and k-d tree from Eq. 10-15; keeps its Steering alive."""

    def __init__(self, steering: Steering, delta: float):
        L = lib()
        h = _vp()
        K = ctypes.c_int()
        _check("sp_svd_reduce", L.sp_svd_reduce(steering.handle, float(delta), 0, ctypes.byref(h), ctypes.byref(K)))
        self._h = h
        self.steering = steering
        self.K = K.value
        self.delta = delta

    @classmethod
    def load(cls, path, materialize_w: bool = False) -> "Basis":
        """sp_load_basis: a basis saved by ``save``; it owns its steering handle."""
        h = _vp()
        K = ctypes.c_int()
        _check("sp_load_basis", lib().sp_load_basis(os.fsencode(path), STEER_MATERIALIZE_W if materialize_w else 0,
                                                    ctypes.byref(h), ctypes.byref(K)))
        self = cls.__new__(cls)
        self._h = h
        self.K = K.value
        sh = _vp()
        _check("sp_basis_steering", lib().sp_basis_steering(h, ctypes.byref(sh)))
        self.steering = Steering._borrowed(sh, materialize_w)
        self.delta = None
        return self

    def save(self, path):
        """sp_save_basis: write the offline results (geometry, K, V, D) to ``path``."""
        _check("sp_save_basis", lib().sp_save_basis(self._h, os.fsencode(path)))

    @property
    def handle(self):
        return self._h

    def sigma2(self) -> np.ndarray:
        n = ctypes.c_int()
        _check("sp_basis_info", lib().sp_basis_info(self._h, None, ctypes.byref(n), None, 0))
        out = np.empty(n.value)
        _check("sp_basis_info", lib().sp_basis_info(self._h, None, None, out.ctypes.data_as(_dp), n.value))
        return out

    def V(self) -> np.ndarray:
        out = np.empty((self.steering.L, self.K), dtype=np.complex128)
        _check("sp_basis_v", lib().sp_basis_v(self._h, out.ctypes.data_as(_dp)))
        return out

    def D(self) -> np.ndarray:
        out = np.empty((self.steering.Q, self.K), dtype=np.complex128)
        _check("sp_basis_d", lib().sp_basis_d(self._h, out.ctypes.data_as(_dp)))
        return out

    def kdtree_info(self) -> dict:
        v = [ctypes.c_int() for _ in range(3)]
        _check("sp_basis_kdtree_info", lib().sp_basis_kdtree_info(self._h, *[ctypes.byref(x) for x in v]))
        return dict(n_nodes=v[0].value, leaf_size=v[1].value, depth=v[2].value)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.sp_basis_destroy(h)
            self._h = None


def build_steering(mic_xyz, dirs, fs, c, N, materialize_w=False) -> Steering:
    return Steering(mic_xyz, dirs, fs, c, N, materialize_w)


def build_steering_nearfield(mic_xyz, src_xyz, fs, c, N, materialize_w=False) -> Steering:
    """Candidate source positions (metres) instead of directions: Eq. 1."""
    return Steering(mic_xyz, src_xyz, fs, c, N, materialize_w, nearfield=True)


def svd_reduce(steering: Steering, delta: float) -> Basis:
    return Basis(steering, delta)


def save_basis(basis: Basis, path) -> None:
    basis.save(path)


def load_basis(path, materialize_w: bool = False) -> Basis:
    return Basis.load(path, materialize_w)


def phat(frames):
    """Eq. 3 / Eq. 7 for every frame: complex64 [T][P*B]."""
    import torch
    _frames(frames, None)
    T, M, B = frames.shape
    X = torch.empty((T, M * (M - 1) // 2 * B), dtype=torch.complex64, device=frames.device)
    _check("sp_phat", lib().sp_phat(_ptr(frames), T, M, B, _ptr(X), _stream()))
    return X


def project(basis: Basis, frames, prec="fp16"):
    """Eq. 12 with fused PHAT: Z = V^H X, complex64 [T][K]."""
    import torch
    _frames(frames, basis.steering)
    Z = torch.empty((frames.shape[0], basis.K), dtype=torch.complex64, device=frames.device)
    _check("sp_project", lib().sp_project(basis.handle, _ptr(frames), frames.shape[0], _prec(prec), _ptr(Z),
                                          _stream()))
    return Z


def localize(basis: Basis, frames, mode="svd_exhaustive", prec="fp16", score=True, proj=True, out=None):
    """Algorithm 1 online steps 1-4.  Returns (idx int32, score float32 | None, proj float32 | None)."""
    import torch
    _frames(frames, basis.steering)
    T = frames.shape[0]
    if out is None:
        idx = torch.empty(T, dtype=torch.int32, device=frames.device)
        sc = torch.empty(T, dtype=torch.float32, device=frames.device) if score else None
        pj = torch.empty(T, dtype=torch.float32, device=frames.device) if proj else None
    else:
        idx, sc, pj = out
    _check("sp_localize", lib().sp_localize(basis.handle, _ptr(frames), T, _mode(mode), _prec(prec), _ptr(idx),
                                            _ptr(sc), _ptr(pj), _stream()))
    return idx, sc, pj


def localize_srp(steering: Steering, frames, score=True):
    """Plain SRP-PHAT (Eq. 5, 6, 9): argmax Re{W X} in FP32; returns (idx, best score)."""
    import torch
    _frames(frames, steering)
    T = frames.shape[0]
    idx = torch.empty(T, dtype=torch.int32, device=frames.device)
    sc = torch.empty(T, dtype=torch.float32, device=frames.device) if score else None
    _check("sp_localize_srp", lib().sp_localize_srp(steering.handle, _ptr(frames), T, _ptr(idx), _ptr(sc),
                                                    _stream()))
    return idx, sc


def localize_host(basis: Basis, frames_host, mode="svd_exhaustive", prec="fp16", score=True, proj=True,
                  chunk_frames=0, out=None):
    """sp_localize from host buffers (pinned CPU tensors); returns CPU tensors."""
    import torch
    if frames_host.is_cuda or frames_host.dtype != torch.complex64 or not frames_host.is_contiguous():
        raise TypeError("frames_host must be a contiguous CPU complex64 tensor")
    T = frames_host.shape[0]
    if out is None:
        pin = frames_host.is_pinned()
        idx = torch.empty(T, dtype=torch.int32, pin_memory=pin)
        sc = torch.empty(T, dtype=torch.float32, pin_memory=pin) if score else None
        pj = torch.empty(T, dtype=torch.float32, pin_memory=pin) if proj else None
    else:
        idx, sc, pj = out
    _check("sp_localize_host", lib().sp_localize_host(basis.handle, _ptr(frames_host), T, _mode(mode), _prec(prec),
                                                      _ptr(idx), _ptr(sc), _ptr(pj), int(chunk_frames),
                                                      _stream()))
    return idx, sc, pj


def localize_noalloc(basis: Basis, frames, prec="fp16", score=True, proj=True, out=None):
    """sp_localize_noalloc: exhaustive FP16/BF16 localisation whose scratch lives in a fixed
    array inside the library (no allocation in the call); T is bounded by that array."""
    import torch
    _frames(frames, basis.steering)
    T = frames.shape[0]
    if out is None:
        idx = torch.empty(T, dtype=torch.int32, device=frames.device)
        sc = torch.empty(T, dtype=torch.float32, device=frames.device) if score else None
        pj = torch.empty(T, dtype=torch.float32, device=frames.device) if proj else None
    else:
        idx, sc, pj = out
    _check("sp_localize_noalloc", lib().sp_localize_noalloc(basis.handle, _ptr(frames), T, _prec(prec), _ptr(idx),
                                                            _ptr(sc), _ptr(pj), _stream()))
    return idx, sc, pj


def kdtree_search(basis: Basis, Z, visits=True):
    """sp_kdtree_search: the k-d tree search (Eq. 15) of given projections Z (device [T][K]
    complex64).  Returns (idx, score, visits) with visits int32 [T][2] (nodes, leaf buckets)
    or None."""
    import torch
    T = Z.shape[0]
    assert Z.dtype == torch.complex64 and Z.is_contiguous() and Z.shape[1] == basis.K
    idx = torch.empty(T, dtype=torch.int32, device=Z.device)
    sc = torch.empty(T, dtype=torch.float32, device=Z.device)
    vi = torch.empty((T, 2), dtype=torch.int32, device=Z.device) if visits else None
    _check("sp_kdtree_search", lib().sp_kdtree_search(basis.handle, _ptr(Z), T, _ptr(idx), _ptr(sc), _ptr(vi),
                                                      _stream()))
    return idx, sc, vi


def n_frames(n_samples: int, N: int, hop: int) -> int:
    """Whole frames of N samples with hop `hop` in n_samples samples."""
    return 0 if n_samples < N else (n_samples - N) // hop + 1


def _samples(x):
    import torch
    assert x.is_cuda and x.dtype == torch.float32 and x.dim() == 2 and x.stride(1) == 1, \
        "samples must be a CUDA float32 [M][S] tensor with contiguous rows"
    return x


def stft(samples, N: int, hop: int, mask=None):
    """sp_stft: sine-window STFT (Section 2) of device samples [M][S] -> frames [T][M][N/2+1]
    complex64; `mask` (uint8 [T][N/2+1], 0 = drop) zeroes bins."""
    import torch
    x = _samples(samples)
    M, S = x.shape
    T = n_frames(S, N, hop)
    out = torch.empty((T, M, N // 2 + 1), dtype=torch.complex64, device=x.device)
    t = ctypes.c_int()
    _check("sp_stft", lib().sp_stft(_ptr(x), M, S, x.stride(0), N, hop, _ptr(mask), _ptr(out), ctypes.byref(t),
                                    _stream()))
    assert t.value == T
    return out


def apply_mask(frames, mask, out=None):
    """sp_apply_mask: frames [T][M][B] complex64 with the bins of mask == 0 zeroed."""
    import torch
    T, M, B = frames.shape
    assert mask.dtype == torch.uint8 and tuple(mask.shape) == (T, B)
    out = torch.empty_like(frames) if out is None else out
    _check("sp_apply_mask", lib().sp_apply_mask(_ptr(frames), T, M, B, _ptr(mask.contiguous()), _ptr(out), _stream()))
    return out


def localize_samples(basis: Basis, samples, hop: int, mode="svd_exhaustive", prec="fp16", mask=None, T=None,
                     score=True, proj=True, out=None):
    """sp_localize_samples: the STFT front end then sp_localize, from device samples [M][S]."""
    import torch
    x = _samples(samples)
    M, S = x.shape
    st = basis.steering
    if T is None:
        T = n_frames(S, st.N, hop)
    if out is None:
        idx = torch.empty(T, dtype=torch.int32, device=x.device)
        sc = torch.empty(T, dtype=torch.float32, device=x.device) if score else None
        pj = torch.empty(T, dtype=torch.float32, device=x.device) if proj else None
    else:
        idx, sc, pj = out
    _check("sp_localize_samples", lib().sp_localize_samples(basis.handle, _ptr(x), S, x.stride(0), hop, _ptr(mask), T,
                                                            _mode(mode), _prec(prec), _ptr(idx), _ptr(sc), _ptr(pj),
                                                            _stream()))
    return idx, sc, pj


def weighted_doa_error(steering: Steering, idx, score, s0, alpha: int) -> float:
    """sp_weighted_doa_error: Section 4's energy-weighted DOA error (Eq. 20) of one configuration."""
    import torch
    assert idx.dtype == torch.int32 and score.dtype == torch.float32 and idx.shape == score.shape
    s0 = np.ascontiguousarray(s0, dtype=np.float64)
    v = ctypes.c_double()
    _check("sp_weighted_doa_error", lib().sp_weighted_doa_error(steering.handle, _ptr(idx.contiguous()),
                                                                _ptr(score.contiguous()), idx.shape[0],
                                                                s0.ctypes.data_as(ctypes.c_void_p), int(alpha),
                                                                ctypes.byref(v), _stream()))
    return v.value


def check_status():
    _check("sp_check_status", lib().sp_check_status(_stream()))


def set_wait_budget(cycles: int):
    _check("sp_set_wait_budget", lib().sp_set_wait_budget(int(cycles)))


def fp32_fma_peak() -> float:
    """sp_fp32_fma_peak: the measured FP32 FMA rate of the current device (TFLOP/s)."""
    v = ctypes.c_double()
    _check("sp_fp32_fma_peak", lib().sp_fp32_fma_peak(ctypes.byref(v)))
    return v.value


def set_tune_cache(path) -> None:
    """sp_set_tune_cache: the JSON file of autotuned batch plans (None disables it)."""
    _check("sp_set_tune_cache", lib().sp_set_tune_cache(None if path is None else str(path).encode()))


def tune_cache_get(key: str):
    """sp_tune_cache_get: the stored shape dict for key, or None."""
    br, tpc, pv, gr, found = (ctypes.c_int() for _ in range(5))
    ms = ctypes.c_float()
    _check("sp_tune_cache_get", lib().sp_tune_cache_get(key.encode(), ctypes.byref(br), ctypes.byref(tpc),
                                                        ctypes.byref(pv), ctypes.byref(ms), ctypes.byref(gr),
                                                        ctypes.byref(found)))
    if not found.value:
        return None
    return dict(branches=br.value, tiles_per_cta=tpc.value, proj_variant=pv.value, ms=ms.value, grouped=gr.value)


def tune_cache_put(key: str, branches: int, tiles_per_cta: int, proj_variant: int, ms: float,
                   grouped: int = 0) -> None:
    _check("sp_tune_cache_put", lib().sp_tune_cache_put(key.encode(), int(branches), int(tiles_per_cta),
                                                        int(proj_variant), float(ms), int(grouped)))


class Proposal:
    """Learned cell proposal over a basis (``sp_proposal_*``); keeps its Basis alive."""

    def __init__(self, basis: Basis, cell_dirs, hidden=(256, 256), seed: int = 0):
        d = np.ascontiguousarray(cell_dirs, dtype=np.float64)
        h = _vp()
        _check("sp_proposal_create", lib().sp_proposal_create(basis.handle, d.ctypes.data_as(_dp), d.shape[0],
                                                              int(hidden[0]), int(hidden[1]), int(seed) & (2**64 - 1),
                                                              ctypes.byref(h)))
        self._h = h
        self.basis = basis
        v = [ctypes.c_int() for _ in range(4)]
        n = ctypes.c_longlong()
        _check("sp_proposal_dims", lib().sp_proposal_dims(h, *[ctypes.byref(x) for x in v], ctypes.byref(n)))
        self.F, self.H1, self.H2, self.C = (x.value for x in v)
        self.n_params = n.value

    @property
    def handle(self):
        return self._h

    def cells(self) -> np.ndarray:
        out = np.empty(self.basis.steering.Q, dtype=np.int32)
        _check("sp_proposal_cells", lib().sp_proposal_cells(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
        return out

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        _check("sp_proposal_get_params", lib().sp_proposal_get_params(
            self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return out

    def set_params(self, theta) -> None:
        t = np.ascontiguousarray(theta, dtype=np.float32)
        if t.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {t.size}")
        _check("sp_proposal_set_params", lib().sp_proposal_set_params(
            self._h, t.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def examples(self, frames, prec="fp16"):
        """Training features [T][F] (float32) and labels [T] (int32) of device frames."""
        import torch
        _frames(frames, self.basis.steering)
        T = frames.shape[0]
        x = torch.empty((T, self.F), dtype=torch.float32, device=frames.device)
        y = torch.empty(T, dtype=torch.int32, device=frames.device)
        _check("sp_proposal_examples", lib().sp_proposal_examples(self._h, _ptr(frames), T, _prec(prec), _ptr(x),
                                                                  _ptr(y), _stream()))
        return x, y

    def forward_f32(self, x):
        import torch
        x = x.contiguous()
        out = torch.empty((x.shape[0], self.C), dtype=torch.float32, device=x.device)
        _check("sp_proposal_forward_f32", lib().sp_proposal_forward_f32(self._h, _ptr(x), x.shape[0], _ptr(out),
                                                                        _stream()))
        return out

    def grad(self, x, labels):
        """(gradient [n_params], mean loss) of the batch, FP32 on the device."""
        import torch
        g = torch.empty(self.n_params, dtype=torch.float32, device=x.device)
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
        _check("sp_proposal_grad", lib().sp_proposal_grad(self._h, _ptr(x.contiguous()), _ptr(labels.contiguous()),
                                                          x.shape[0], _ptr(g), _ptr(loss), _stream()))
        return g, loss

    def train_step(self, x, labels, rows=None, lr=1e-3, loss=None):
        n = x.shape[0] if rows is None else rows.shape[0]
        _check("sp_proposal_train_step", lib().sp_proposal_train_step(self._h, _ptr(x), _ptr(labels), _ptr(rows), n,
                                                                      float(lr), _ptr(loss), _stream()))

    def train(self, x, labels, epochs=10, batch=512, lr=1e-3, seed=0):
        """Adam over shuffled mini-batches of (x, labels); returns the mean loss per epoch."""
        import torch
        T = x.shape[0]
        rng = np.random.default_rng(seed)
        losses = torch.empty((epochs, (T + batch - 1) // batch), dtype=torch.float32, device=x.device)
        for e in range(epochs):
            perm = torch.from_numpy(rng.permutation(T).astype(np.int32)).to(x.device)
            for i, b0 in enumerate(range(0, T, batch)):
                rows = perm[b0:b0 + batch]
                self.train_step(x, labels, rows=rows, lr=lr, loss=losses[e, i:i + 1])
        return losses.mean(dim=1).cpu().numpy()

    def infer(self, Z, zn2, logits=False):
        """Tensor-core inference from Z [T][K] complex64 and ||Z||^2 [T]: (top8, conf, logits|None)."""
        import torch
        T = Z.shape[0]
        top = torch.empty((T, 8), dtype=torch.int32, device=Z.device)
        conf = torch.empty(T, dtype=torch.float32, device=Z.device)
        lg = torch.empty((T, self.C), dtype=torch.float32, device=Z.device) if logits else None
        _check("sp_proposal_infer", lib().sp_proposal_infer(self._h, _ptr(Z.contiguous()), _ptr(zn2.contiguous()), T,
                                                            _ptr(lg), _ptr(top), _ptr(conf), _stream()))
        return top, conf, lg

    def localize(self, frames, prec="fp16", n_top=4, theta=0.5, score=True, proj=True, fallback=True):
        """sp_localize_learned: returns (idx, score|None, proj|None, fallback|None)."""
        import torch
        _frames(frames, self.basis.steering)
        T = frames.shape[0]
        idx = torch.empty(T, dtype=torch.int32, device=frames.device)
        sc = torch.empty(T, dtype=torch.float32, device=frames.device) if score else None
        pj = torch.empty(T, dtype=torch.float32, device=frames.device) if proj else None
        fb = torch.empty(T, dtype=torch.int32, device=frames.device) if fallback else None
        _check("sp_localize_learned", lib().sp_localize_learned(self._h, _ptr(frames), T, _prec(prec), int(n_top),
                                                                float(theta), _ptr(idx), _ptr(sc), _ptr(pj), _ptr(fb),
                                                                _stream()))
        return idx, sc, pj, fb

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.sp_proposal_destroy(h)
            self._h = None


def _ptr_array(items):
    arr = (ctypes.c_void_p * len(items))(*[None if t is None else t.data_ptr() for t in items])
    return arr


class Batch:
    """A batch plan (``sp_batch_*``): many streams, one CUDA-graph launch per ``run()``.

    ``frames`` is a list of CUDA complex64 tensors [T_i][M_i][B_i] (kept alive and read at
    every run); results land in ``self.idx`` / ``self.score`` / ``self.proj`` (lists of
    tensors, one per stream)."""

    def __init__(self, bases, frames, mode="svd_exhaustive", prec="fp16", score=True, proj=True, autotune=False,
                 tune_kernels=False, group=False):
        import torch
        n = len(bases)
        if len(frames) != n:
            raise ValueError("one frame tensor per basis")
        for b, f in zip(bases, frames):
            _frames(f, b.steering)
        self.bases, self.frames = list(bases), list(frames)
        T = [int(f.shape[0]) for f in frames]
        self.idx = [torch.empty(t, dtype=torch.int32, device=f.device) for t, f in zip(T, frames)]
        self.score = [torch.empty(t, dtype=torch.float32, device=f.device) for t, f in zip(T, frames)] if score else None
        self.proj = [torch.empty(t, dtype=torch.float32, device=f.device) for t, f in zip(T, frames)] if proj else None
        bh = (ctypes.c_void_p * n)(*[b.handle.value for b in bases])
        Ta = (ctypes.c_int * n)(*T)
        h = _vp()
        _check("sp_batch_create", lib().sp_batch_create(
            n, bh, _ptr_array(frames), Ta, _mode(mode), _prec(prec), _ptr_array(self.idx),
            _ptr_array(self.score) if score else None, _ptr_array(self.proj) if proj else None,
            (1 if autotune else 0) | (2 if tune_kernels else 0) | (4 if group else 0), _stream(), ctypes.byref(h)))
        self._h = h

    def run(self):
        _check("sp_batch_run", lib().sp_batch_run(self._h, _stream()))

    def info(self) -> dict:
        br, tpc, pv, nf, fc, gr, ng = (ctypes.c_int() for _ in range(7))
        ms = ctypes.c_float()
        _check("sp_batch_info", lib().sp_batch_info(self._h, ctypes.byref(br), ctypes.byref(tpc), ctypes.byref(pv),
                                                    ctypes.byref(ms), ctypes.byref(nf), ctypes.byref(fc),
                                                    ctypes.byref(gr), ctypes.byref(ng)))
        return dict(branches=br.value, tiles_per_cta=tpc.value, proj_variant=pv.value, ms=ms.value,
                    n_fp32=nf.value, from_cache=bool(fc.value), grouped=bool(gr.value), n_groups=ng.value)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.sp_batch_destroy(h)
            self._h = None


def localize_batched(bases, frames, mode="svd_exhaustive", prec="fp16"):
    """sp_localize_batched: returns (idx list, score list, proj list)."""
    import torch
    n = len(bases)
    T = [int(f.shape[0]) for f in frames]
    idx = [torch.empty(t, dtype=torch.int32, device=f.device) for t, f in zip(T, frames)]
    sc = [torch.empty(t, dtype=torch.float32, device=f.device) for t, f in zip(T, frames)]
    pj = [torch.empty(t, dtype=torch.float32, device=f.device) for t, f in zip(T, frames)]
    bh = (ctypes.c_void_p * n)(*[b.handle.value for b in bases])
    _check("sp_localize_batched", lib().sp_localize_batched(
        n, bh, _ptr_array(frames), (ctypes.c_int * n)(*T), _mode(mode), _prec(prec), _ptr_array(idx),
        _ptr_array(sc), _ptr_array(pj), _stream()))
    return idx, sc, pj
