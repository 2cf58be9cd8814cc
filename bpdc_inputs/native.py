"""Builds and calls the native input-construction helpers (trivial_errors.c)
with gcc; the library lands in bpdc_inputs/_build/ (rebuilt when stale)."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "trivial_errors.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libtrivial.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        p32 = ctypes.POINTER(ctypes.c_int32)
        lib.trivial_errors.restype = ctypes.c_int64
        lib.trivial_errors.argtypes = [ctypes.c_int] * 4 + [p32] * 4 + [ctypes.POINTER(ctypes.c_uint64), p32,
                                                                       ctypes.c_int64]
        _lib = lib
    return _lib


def trivial_errors(H, O, w: int, cap: int = 4_000_000) -> set:
    """All sets of at most w columns with H 1_S = 0 and O 1_S = 0 whose support
    is connected through shared rows of H (every such set for the BB detector
    models at w <= 5), as sorted column tuples."""
    Hr = sp.csr_matrix(H, dtype=np.uint8)
    Hr.sort_indices()
    Hc = sp.csc_matrix(Hr)
    Hc.sort_indices()
    Od = np.asarray(sp.csr_matrix(O).toarray(), dtype=np.uint64)
    K = Od.shape[0]
    assert K <= 64
    obs = (Od * (np.uint64(1) << np.arange(K, dtype=np.uint64))[:, None]).sum(axis=0).astype(np.uint64)
    rp = np.ascontiguousarray(Hr.indptr, dtype=np.int32)
    rc = np.ascontiguousarray(Hr.indices, dtype=np.int32)
    cp = np.ascontiguousarray(Hc.indptr, dtype=np.int32)
    cr = np.ascontiguousarray(Hc.indices, dtype=np.int32)
    obs = np.ascontiguousarray(obs)
    out = np.empty((cap, w), dtype=np.int32)
    p32 = ctypes.POINTER(ctypes.c_int32)
    n = _load().trivial_errors(Hr.shape[0], Hr.shape[1], K, w, rp.ctypes.data_as(p32), rc.ctypes.data_as(p32),
                               cp.ctypes.data_as(p32), cr.ctypes.data_as(p32),
                               obs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), out.ctypes.data_as(p32), cap)
    if n < 0:
        raise RuntimeError("trivial-error search: output capacity exceeded")
    return {tuple(sorted(int(c) for c in row if c >= 0)) for row in out[:n]}
