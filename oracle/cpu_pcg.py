"""ctypes wrapper of cpu_pcg.c: the CPU block PCG baseline (test and
measurement infrastructure; the GPU library never loads it).

build() compiles cpu_pcg.c with gcc and OpenMP next to this file;
block_pcg(A, B, ...) runs the Sec. 2.3.1 iteration (diagonal-preconditioned
CG, one column per electrode, App. A.4) on a scipy CSR matrix and a dense
node-major right-hand side block.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpu_pcg.c")
LIB = os.path.join(HERE, "_cpu_pcg.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        subprocess.run(["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", "-o", LIB, SRC, "-lm"], check=True)
    return LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        f = _lib.zi_cpu_block_pcg
        f.restype = ctypes.c_int
        f.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                      ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                      ctypes.c_void_p, ctypes.c_int]
    return _lib


def block_pcg(A, B, tol=1e-10, maxit=100000, precond=0, threads=0):
    """T (n x L), per-column iterations, and the largest count.  precond 0:
    Jacobi (a_ii), 1: lumped diagonal (sum_j |a_ij|).  threads 0: OpenMP's
    default."""
    A = A.tocsr()
    n = A.shape[0]
    rowptr = np.ascontiguousarray(A.indptr, dtype=np.int32)
    colind = np.ascontiguousarray(A.indices, dtype=np.int32)
    vals = np.ascontiguousarray(A.data, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    L = B.shape[1]
    T = np.zeros((n, L))
    iters = np.zeros(L, dtype=np.int32)
    k = _load().zi_cpu_block_pcg(n, rowptr.ctypes.data, colind.ctypes.data, vals.ctypes.data, L, B.ctypes.data,
                                 float(tol), int(maxit), int(precond), T.ctypes.data, iters.ctypes.data,
                                 int(threads))
    if k < 0:
        raise RuntimeError("cpu block PCG failed")
    return T, iters, k
