"""ctypes wrapper of the oracle's plain-C ILU(0) (test infrastructure only)."""
import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, 'ilu0.c')
_LIB = os.path.join(_HERE, '_ilu0.so')
_lib = None


def build():
    """Compile ilu0.c into oracle/_ilu0.so (plain C, no machine-specific flags)."""
    subprocess.check_call(['gcc', '-O2', '-fPIC', '-shared', '-o', _LIB, _SRC])


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        lib.ilu0_factor.argtypes = [ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_double), P(ctypes.c_int)]
        lib.ilu0_factor.restype = ctypes.c_int
        lib.ilu0_solve.argtypes = [ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_double), P(ctypes.c_int),
                                   P(ctypes.c_double), P(ctypes.c_double)]
        lib.ilu0_solve.restype = None
        _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


class ILU0:
    """ILU(0) factors of a square CSR matrix with sorted indices and explicit diagonal."""

    def __init__(self, A: sp.csr_matrix):
        A = sp.csr_matrix(A, copy=True)
        A.has_sorted_indices = False
        A.sort_indices()
        self.n = A.shape[0]
        self.indptr = np.ascontiguousarray(A.indptr, dtype=np.int32)
        self.indices = np.ascontiguousarray(A.indices, dtype=np.int32)
        self.a = np.ascontiguousarray(A.data, dtype=np.float64)
        self.diag = np.empty(self.n, dtype=np.int32)
        rc = _load().ilu0_factor(self.n, _p(self.indptr, ctypes.c_int), _p(self.indices, ctypes.c_int),
                                 _p(self.a, ctypes.c_double), _p(self.diag, ctypes.c_int))
        if rc != 0:
            raise ZeroDivisionError('ILU(0): zero or missing pivot in row %d' % (rc - 1))

    def solve(self, b):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.empty_like(b)
        _load().ilu0_solve(self.n, _p(self.indptr, ctypes.c_int), _p(self.indices, ctypes.c_int),
                           _p(self.a, ctypes.c_double), _p(self.diag, ctypes.c_int),
                           _p(b, ctypes.c_double), _p(x, ctypes.c_double))
        return x
