"""Loader for the oracle's C part (test infrastructure only).

``build_native()`` compiles ``topk.c`` with gcc into ``_oracle_topk.so`` next
to this file; ``ivf_topk`` calls it through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "topk.c")
_LIB = os.path.join(_HERE, "_oracle_topk.so")
_lib = None


def build_native(force: bool = False) -> str:
    """Compile topk.c (plain C, -O2, portable flags) if it is out of date."""
    if force or not os.path.exists(_LIB) or \
            os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-pthread", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build_native()
        lib = ctypes.CDLL(_LIB)
        lib.oracle_ivf_topk.restype = ctypes.c_int
        lib.oracle_ivf_topk.argtypes = [
            ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def ivf_topk(X, Q, ptr, rows, probes, k, threads: int = 0):
    """FP64 brute-force top-k of each query over the union of its probed lists.

    probes: list of int arrays (or a 2-D int array); k: int array per query.
    Returns (ids int64 [nq, k_max], dists float64 [nq, k_max]).
    """
    lib = _load()
    X = np.ascontiguousarray(X, dtype=np.float32)
    Q = np.ascontiguousarray(Q, dtype=np.float32)
    nq, d = Q.shape
    ptr = np.ascontiguousarray(ptr, dtype=np.int64)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    if isinstance(probes, np.ndarray) and probes.ndim == 2:
        P = np.ascontiguousarray(probes, dtype=np.int32)
        npr = np.full(nq, P.shape[1], dtype=np.int32)
    else:
        width = max(1, max((len(p) for p in probes), default=1))
        P = np.zeros((nq, width), dtype=np.int32)
        npr = np.zeros(nq, dtype=np.int32)
        for i, p in enumerate(probes):
            P[i, :len(p)] = p
            npr[i] = len(p)
    k = np.ascontiguousarray(np.broadcast_to(np.asarray(k), (nq,)),
                             dtype=np.int32)
    k_max = int(k.max()) if nq else 1
    out_i = np.empty((nq, k_max), dtype=np.int64)
    out_d = np.empty((nq, k_max), dtype=np.float64)
    if threads <= 0:
        threads = os.cpu_count() or 1
    rc = lib.oracle_ivf_topk(_ptr(X), d, _ptr(Q), nq, _ptr(ptr), _ptr(rows),
                             _ptr(P), P.shape[1], _ptr(npr), _ptr(k), k_max,
                             _ptr(out_i), _ptr(out_d), threads)
    if rc != 0:
        raise MemoryError("oracle_ivf_topk failed")
    return out_i, out_d
