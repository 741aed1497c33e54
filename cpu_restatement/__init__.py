"""CPU restatement of the paper's Newton-step design (a CPU measurement
baseline, not the product and not the oracle).

``kkt_pcg_cpu.cpp`` applies the doubly augmented KKT matrix of Eq. (9)
matrix-free in FP64 with OpenMP and solves it by Jacobi-PCG, as the paper's
C++/OpenBLAS prototype does on a CPU (section 3.2, section 4).  It shares no
code with the GPU library or the oracle.  ``bench.py`` times it on the host
cores for PCG iterations per second; ``tests/test_cpu_restatement.py`` checks
it against the oracle.  Built with g++ -O3 -fopenmp into this folder.
"""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "kkt_pcg_cpu.cpp")
LIB = os.path.join(HERE, "libkkt_cpu.so")
_lib = None


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        raise RuntimeError("no C++ compiler for the CPU restatement")
    tmp = LIB + ".tmp"
    r = subprocess.run([cxx, "-O3", "-fopenmp", "-shared", "-fPIC", "-std=c++17", SRC, "-o", tmp],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("g++ failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


def load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(LIB)
        P = C.c_void_p
        I64 = C.c_int64
        common = [I64, I64, P, P, P, P, I64, P, P, P, I64, P, I64, P, P, P]
        lib.cpu_kkt_apply.restype = C.c_int
        lib.cpu_kkt_apply.argtypes = common + [P, P]
        lib.cpu_kkt_pcg.restype = C.c_int
        lib.cpu_kkt_pcg.argtypes = common + [P, P, C.c_double, C.c_int, P, C.POINTER(C.c_double)]
        lib.cpu_threads.restype = C.c_int
        _lib = lib
    return _lib


class System:
    """The Eq. (9) system of a CSR least-squares QP with general CSR rows
    (H = P' diag(w2) P, B = [A_L; -A_U]) at one iterate: arrays held in the
    layout the C++ code takes."""

    def __init__(self, P, w2, A, L, U, dg, D):
        P = P.tocsr()
        A = A.tocsr()
        self.n = P.shape[1]
        self.nP = P.shape[0]
        self.m = A.shape[0]
        self.prow = np.ascontiguousarray(P.indptr, dtype=np.int64)
        self.pcol = np.ascontiguousarray(P.indices, dtype=np.int32)
        self.pval = np.ascontiguousarray(P.data, dtype=np.float64)
        self.w2 = np.ascontiguousarray(w2, dtype=np.float64)
        self.arow = np.ascontiguousarray(A.indptr, dtype=np.int64)
        self.acol = np.ascontiguousarray(A.indices, dtype=np.int32)
        self.aval = np.ascontiguousarray(A.data, dtype=np.float64)
        self.L = np.ascontiguousarray(L, dtype=np.int32)
        self.U = np.ascontiguousarray(U, dtype=np.int32)
        self.dg = np.ascontiguousarray(dg, dtype=np.float64)
        self.D = np.ascontiguousarray(D, dtype=np.float64)
        self.N = self.n + len(self.L) + len(self.U)
        self.nnzP = int(P.nnz)
        self.nnzA = int(A.nnz)

    def _args(self):
        p = lambda a: a.ctypes.data_as(C.c_void_p)
        return [self.n, self.nP, p(self.prow), p(self.pcol), p(self.pval), p(self.w2), self.m,
                p(self.arow), p(self.acol), p(self.aval), len(self.L), p(self.L), len(self.U),
                p(self.U), p(self.dg), p(self.D)]

    def apply(self, v):
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.zeros(self.N)
        load().cpu_kkt_apply(*self._args(), v.ctypes.data_as(C.c_void_p),
                             out.ctypes.data_as(C.c_void_p))
        return out

    def pcg(self, diag, rhs, tol=1e-7, maxit=5000):
        diag = np.ascontiguousarray(diag, dtype=np.float64)
        rhs = np.ascontiguousarray(rhs, dtype=np.float64)
        sol = np.zeros(self.N)
        rel = C.c_double()
        it = load().cpu_kkt_pcg(*self._args(), diag.ctypes.data_as(C.c_void_p),
                                rhs.ctypes.data_as(C.c_void_p), float(tol), int(maxit),
                                sol.ctypes.data_as(C.c_void_p), C.byref(rel))
        return sol, it, rel.value

    def bytes_per_apply(self):
        """Bytes one apply reads: P twice (row dots, then the transposed
        scatter: 8 B value + 4 B column per nonzero, 8 B row pointer per row),
        w2, and A twice."""
        return (2 * (self.nnzP * 12 + (self.nP + 1) * 8) + self.nP * 8
                + 2 * (self.nnzA * 12 + (self.m + 1) * 8))


def threads() -> int:
    return int(load().cpu_threads())
