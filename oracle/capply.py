"""ctypes binding of ``capply.c`` (oracle, test infrastructure only).

``build()`` compiles the C file with gcc (OpenMP when available) into
``oracle/_build/liboracle_capply.so``; ``bf_apply_c`` / ``bf_adjoint_c`` run the
FP64 loops of ``capply.c`` on a ``ButterflyFactors`` and a host vector.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from bfinputs.factors import ButterflyFactors

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "capply.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle_capply.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile capply.c (gcc -O2, -fopenmp if it links) and return the .so path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", _LIB + ".tmp"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_bf_apply.restype = ctypes.c_int
        lib.oracle_bf_apply.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_long, ctypes.c_int]
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    """Threads the OpenMP loops of capply.c use."""
    return int(_load().oracle_num_threads())


class PreparedFactors:
    """FP64 contiguous copies of the factors, kept alive for repeated C calls."""

    def __init__(self, F: ButterflyFactors):
        F64 = F.astype(np.complex128)
        self.F = F64
        self.h_arr = (ctypes.c_void_p * max(1, len(F64.H)))(*[a.ctypes.data for a in F64.H])
        self.g_arr = (ctypes.c_void_p * max(1, len(F64.G)))(*[a.ctypes.data for a in F64.G])


def _run(P: PreparedFactors, x: np.ndarray, adjoint: bool) -> np.ndarray:
    F = P.F
    x = np.asarray(x)
    squeeze = x.ndim == 1
    cols = np.ascontiguousarray(x.reshape(F.N, -1).T, dtype=np.complex128)   # (nrhs, N)
    out = np.empty_like(cols)
    rc = _load().oracle_bf_apply(F.L, F.n0, F.r, F.VL.ctypes.data, P.h_arr, F.S.ctypes.data,
                                 P.g_arr, F.UL.ctypes.data, cols.ctypes.data, out.ctypes.data,
                                 cols.shape[0], 1 if adjoint else 0)
    if rc != 0:
        raise RuntimeError("oracle_bf_apply failed")
    res = out.T
    return res[:, 0].copy() if squeeze else np.ascontiguousarray(res)


def bf_apply_c(F, g: np.ndarray) -> np.ndarray:
    """u = K_bf g by the C loops (``F``: ButterflyFactors or PreparedFactors)."""
    P = F if isinstance(F, PreparedFactors) else PreparedFactors(F)
    return _run(P, g, False)


def bf_adjoint_c(F, f: np.ndarray) -> np.ndarray:
    """K_bf^* f by the C loops."""
    P = F if isinstance(F, PreparedFactors) else PreparedFactors(F)
    return _run(P, f, True)
