"""CPU FP64 oracle for the Hermitian-definite generalized eigenproblem.

TEST INFRASTRUCTURE ONLY.  The oracle is a plain C implementation
(``oracle.c``) of the paper's Algorithm 1 (Cholesky, reduction to the
standard problem, standard eigensolver, back-substitution) around
Algorithm 2 with a single stage (Section 4.1: Householder tridiagonalisation,
a tridiagonal eigensolver, back-transformation).  Only the tests, the smoke
check and the benchmark's CPU-baseline leg may load it; the CUDA library
never does, and the two share no code.

Parity status per function (what pins each one is in ``tests/test_oracle.py``):
  potrf, hegst, hetrd, steqr, unmtr, trsm_lh, hegv -- all pinned (brute force
  at n <= 8, closed forms, constructed spectra, residual ratios, an
  independent library cross-check, reconstructions).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liborc.so (plain gcc, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def bind(path):
    """Load a compiled oracle library and declare its signatures."""
    lib = ctypes.CDLL(path)
    P, I = ctypes.c_void_p, ctypes.c_int
    lib.orc_num_threads.restype = I
    lib.orc_potrf.argtypes = [I, P, I]
    lib.orc_potrf.restype = I
    lib.orc_hegst.argtypes = [I, P, I, P, I]
    lib.orc_hetrd.argtypes = [I, P, I, P, P, P, I, P]
    lib.orc_steqr.argtypes = [I, P, P, P, I]
    lib.orc_steqr.restype = I
    lib.orc_sort_eig.argtypes = [I, P, P, I]
    lib.orc_unmtr.argtypes = [I, I, P, I, P, P, I]
    lib.orc_trsm_lh.argtypes = [I, I, P, I, P, I]
    lib.orc_hegv.argtypes = [I, P, I, P, I, I, I, P, P, I]
    lib.orc_hegv.restype = I
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = bind(_LIB)
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _zmat(a):
    return np.array(a, dtype=np.complex128, order="F", copy=True)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def potrf(B):
    """Algorithm 1 step 1: returns (L, info); L lower with zero upper part."""
    B = _zmat(B)
    n = B.shape[0]
    info = _load().orc_potrf(n, _p(B), max(n, 1))
    return np.tril(B), int(info)


def hegst(A, L):
    """Algorithm 1 step 2: full Hermitian A' = L^{-1} A L^{-H} (A lower read)."""
    A = _zmat(A)
    L = _zmat(L)
    n = A.shape[0]
    _load().orc_hegst(n, _p(A), max(n, 1), _p(L), max(n, 1))
    return A


def hetrd(A):
    """One-stage Householder tridiagonalisation of the FULL Hermitian A.

    Returns (d, e, V, tau): A = Q T Q^H with Q = H_0 ... H_{n-2},
    H_k = I - tau_k V[:,k] V[:,k]^H."""
    A = _zmat(A)
    n = A.shape[0]
    d = np.zeros(n)
    e = np.zeros(max(n - 1, 1))
    V = np.zeros((n, n), dtype=np.complex128, order="F")
    tau = np.zeros(max(n, 1), dtype=np.complex128)
    _load().orc_hetrd(n, _p(A), max(n, 1), _p(d), _p(e), _p(V), max(n, 1), _p(tau))
    return d, e[: max(n - 1, 0)], V, tau[:n]


def steqr(d, e, Z=None):
    """Implicit symmetric QR on tridiagonal (d, e); returns (w, Z, info), unsorted."""
    d = np.array(d, dtype=np.float64, copy=True)
    n = d.shape[0]
    e = np.ascontiguousarray(np.array(e, dtype=np.float64).reshape(-1)[: max(n - 1, 0)])
    e = np.concatenate([e, [0.0]])
    if Z is None:
        Z = np.eye(n, order="F")
    Z = np.array(Z, dtype=np.float64, order="F", copy=True)
    info = _load().orc_steqr(n, _p(d), _p(e), _p(Z), max(n, 1))
    return d, Z, int(info)


def sort_eig(w, Z):
    w = np.array(w, dtype=np.float64, copy=True)
    Z = np.array(Z, dtype=np.float64, order="F", copy=True)
    n = w.shape[0]
    _load().orc_sort_eig(n, _p(w), _p(Z), max(n, 1))
    return w, Z


def unmtr(V, tau, Y):
    """Y := Q Y with Q = H_0 ... H_{n-2} (Algorithm 2 step 3)."""
    V = _zmat(V)
    Y = _zmat(Y)
    tau = np.array(tau, dtype=np.complex128, copy=True)
    n, m = Y.shape
    _load().orc_unmtr(n, m, _p(V), max(n, 1), _p(tau), _p(Y), max(n, 1))
    return Y


def trsm_lh(L, Y):
    """X = L^{-H} Y (Algorithm 1 step 4)."""
    L = _zmat(L)
    X = _zmat(Y)
    n, m = X.shape
    _load().orc_trsm_lh(n, m, _p(L), max(n, 1), _p(X), max(n, 1))
    return X


def hegv(A, B, il=1, iu=None):
    """Eigenpairs il..iu (1-based inclusive) of A x = lambda B x.

    Returns (w, X, info); X is B-orthonormal, w ascending."""
    A = _zmat(A)
    B = _zmat(B)
    n = A.shape[0]
    if iu is None:
        iu = n
    m = max(iu - il + 1, 0)
    w = np.zeros(max(m, 1))
    X = np.zeros((n, max(m, 1)), dtype=np.complex128, order="F")
    info = _load().orc_hegv(n, _p(A), max(n, 1), _p(B), max(n, 1), il, iu, _p(w), _p(X), max(n, 1))
    return w[:m], X[:, :m], int(info)
