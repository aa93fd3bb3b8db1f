"""ctypes loader for the C oracle (operator apply + unpreconditioned CG).

Test infrastructure only. ``build()`` compiles ``h1w_oracle.c`` with gcc and
OpenMP into ``_build/libh1w_oracle.so`` beside this file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "h1w_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libh1w_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc -O2 -fopenmp -shared)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"],
                       check=True)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I = ctypes.c_int64
        D = ctypes.c_double
        _lib.h1wo_apply.argtypes = [I, P, P, P, D, I, P, P, P, P]
        _lib.h1wo_apply.restype = None
        _lib.h1wo_cg.argtypes = [I, P, P, P, D, I, P, P, D, I, P, P, P, P, P, P]
        _lib.h1wo_cg.restype = I
        _lib.h1wo_threads.restype = ctypes.c_int
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class CsrOperator:
    """Holds contiguous CSR arrays of K + M and a dense row-major J."""

    def __init__(self, A: sp.csr_matrix, alpha: float, J: np.ndarray):
        A = A.tocsr()
        self.N = A.shape[0]
        self.indptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
        self.indices = np.ascontiguousarray(A.indices, dtype=np.int64)
        self.data = np.ascontiguousarray(A.data, dtype=np.float64)
        self.alpha = float(alpha)
        self.J = np.ascontiguousarray(J, dtype=np.float64)
        self.m = self.J.shape[0]
        self.w = np.zeros(max(self.m, 1))

    def apply(self, p: np.ndarray) -> np.ndarray:
        p = np.ascontiguousarray(p, dtype=np.float64)
        q = np.empty(self.N)
        lib().h1wo_apply(self.N, _ptr(self.indptr), _ptr(self.indices), _ptr(self.data),
                         self.alpha, self.m, _ptr(self.J), _ptr(p), _ptr(q), _ptr(self.w))
        return q

    def cg(self, b: np.ndarray, rtol: float, maxit: int):
        """Returns (x, iterations, recursive relative residual)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x, r, p, q = (np.empty(self.N) for _ in range(4))
        rel = ctypes.c_double(0.0)
        it = lib().h1wo_cg(self.N, _ptr(self.indptr), _ptr(self.indices), _ptr(self.data), self.alpha,
                           self.m, _ptr(self.J), _ptr(b), rtol, maxit, _ptr(x), _ptr(r), _ptr(p),
                           _ptr(q), _ptr(self.w), ctypes.byref(rel))
        return x, int(it), rel.value


def threads() -> int:
    return int(lib().h1wo_threads())
