"""ctypes loader for oracle/csr_ref.c (TEST INFRASTRUCTURE ONLY).

Compiles the plain-C FP64 CSR operator with gcc into oracle/_build/ on first
use (or when build() of the repository has already done so).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csr_ref.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "libcsr_oracle.so")
_lib = None


def build() -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        f = lib.oracle_csr_gram_apply
        f.restype = ctypes.c_double
        f.argtypes = [ctypes.c_int64, ctypes.c_int64] + [ctypes.c_void_p] * 5
        _lib = lib
    return _lib


def csr_gram_apply(row_ptr, col_idx, values, v, w=None, r0: int = 0, r1: int | None = None):
    """w += A[r0:r1]^T (A[r0:r1] v); returns (w, ||A[r0:r1] v||^2), FP64."""
    lib = _load()
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    values = np.ascontiguousarray(values, dtype=np.float32)
    v = np.ascontiguousarray(v, dtype=np.float64)
    if r1 is None:
        r1 = row_ptr.shape[0] - 1
    if w is None:
        w = np.zeros(v.shape[0], dtype=np.float64)
    ss = lib.oracle_csr_gram_apply(r0, r1, row_ptr.ctypes.data, col_idx.ctypes.data,
                                   values.ctypes.data, v.ctypes.data, w.ctypes.data)
    return w, ss
