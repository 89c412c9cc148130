"""Writes the oracle's FP64 basis in the library's basis-file layout (the 80-byte header,
FP64 arrays, FNV-1a 64 checksum documented with sp_save_basis), so that a step of the CUDA
path can be fed the oracle's own V and D through sp_load_basis."""
import struct

import numpy as np


def write(path, mic, dirs, fs, c, N, delta, ob):
    mic = np.ascontiguousarray(mic, dtype=np.float64)
    dirs = np.ascontiguousarray(dirs, dtype=np.float64)
    K = int(ob["K"])
    sig = np.ascontiguousarray(ob["sigma2"], dtype=np.float64)
    V = np.ascontiguousarray(ob["V"], dtype=np.complex128)
    D = np.ascontiguousarray(ob["D"], dtype=np.complex128)
    body = b"".join(a.tobytes() for a in (mic, dirs, sig, V.view(np.float64), D.view(np.float64)))
    hdr = b"SVDPHAT1" + struct.pack("<II6i3dQQ", 1, 80, mic.shape[0], dirs.shape[0], int(N), K, sig.size, 0,
                                    float(fs), float(c), float(delta), len(body), 0)
    h = 1469598103934665603                    # FNV-1a 64 over every preceding byte
    data = hdr + body
    arr = np.frombuffer(data, dtype=np.uint8)
    for byte in arr.tolist():
        h = ((h ^ byte) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    with open(path, "wb") as f:
        f.write(data + struct.pack("<Q", h))
