"""OpenMP build of the oracle's Jacobi-PCG (``oracle/pcg_omp.c``).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: used by ``tests/``
and by the CPU-baseline leg of ``bench.py`` to time the oracle's PCG on one
thread and on every host core.  The recurrence is the one of
``oracle.pirmcut.pcg_jacobi`` (Section 3.1), written out in C; the C file is
compiled here with gcc (``build()``), never by or into the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pcg_omp.c")
LIB = os.path.join(HERE, "libpcg_omp.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile pcg_omp.c into oracle/libpcg_omp.so (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"],
                       check=True)
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.oracle_pcg_jacobi.restype = ctypes.c_int
        _lib.oracle_pcg_jacobi.argtypes = [
            ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, ctypes.c_int,
            ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]
        _lib.oracle_max_threads.restype = ctypes.c_int
    return _lib


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def pcg_jacobi(A, b, x0=None, tol=1e-10, maxit=20000, threads=0):
    """Jacobi-PCG on the CSR matrix A (same recurrence and stopping test as
    ``oracle.pirmcut.pcg_jacobi``), ``threads`` OpenMP threads (0 = the
    OpenMP default).  Returns (x, iterations, ||r||/||b||)."""
    A = sp.csr_matrix(A)
    indptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
    indices = np.ascontiguousarray(A.indices, dtype=np.int32)
    data = np.ascontiguousarray(A.data, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    it = ctypes.c_int64(0)
    rel = ctypes.c_double(0.0)
    st = lib().oracle_pcg_jacobi(A.shape[0], indptr.ctypes.data, indices.ctypes.data,
                                 data.ctypes.data, b.ctypes.data, x.ctypes.data, float(tol),
                                 int(maxit), int(threads), ctypes.byref(it), ctypes.byref(rel))
    if st == 1:
        raise MemoryError("pcg_omp: out of memory")
    if st == 2:
        raise ValueError("pcg_omp: zero on the diagonal")
    return x, int(it.value), float(rel.value)
