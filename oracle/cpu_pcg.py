"""Multi-core CPU baseline of the oracle's solve.

TEST INFRASTRUCTURE ONLY (benchmark CPU baseline and its pin in tests/).
Loads oracle/cpu_pcg.c -- Jacobi PCG (Algorithm 1, last step) on the explicit
CSR operator of eq. GF with OpenMP row-parallel products -- compiled by gcc
into oracle/_build/ (by the package's build entry point, or here on first use).
Same recurrences as oracle.solve.pcg; pinned against it and against
manufactured solutions in tests/test_oracle_cpu_pcg.py.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpu_pcg.c")
LIB = os.path.join(HERE, "_build", "libcpu_pcg.so")
GCC = ["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", SRC, "-o", LIB, "-lm"]


def build():
    """Compile the C baseline if it is missing or older than its source."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        subprocess.run(GCC, check=True)
    return LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        lib.pcg_csr.restype = C.c_int
        lib.pcg_csr.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                C.c_int, C.c_int, C.c_void_p]
        lib.pcg_threads.restype = C.c_int
        _lib = lib
    return _lib


def threads():
    """OpenMP threads the solver uses by default."""
    return int(_load().pcg_threads())


def pcg(L, b, D, tol=1e-14, max_iter=10000, n_threads=0):
    """(x, iterations) for the sparse matrix L (complex128), right-hand side b
    and Jacobi diagonal D; n_threads = 0 keeps the OpenMP default."""
    lib = _load()
    L = L.tocsr()
    n = L.shape[0]
    ip = np.ascontiguousarray(L.indptr.astype(np.int64))
    ix = np.ascontiguousarray(L.indices.astype(np.int32))
    v = np.ascontiguousarray(L.data.astype(np.complex128))
    bb = np.ascontiguousarray(np.asarray(b, np.complex128))
    DD = np.ascontiguousarray(np.asarray(D, np.float64))
    x = np.zeros(n, np.complex128)
    it = lib.pcg_csr(n, ip.ctypes.data, ix.ctypes.data, v.ctypes.data, bb.ctypes.data, DD.ctypes.data, float(tol),
                     int(max_iter), int(n_threads), x.ctypes.data)
    if it < 0:
        raise MemoryError("cpu_pcg: work vector allocation failed")
    return x, it
