"""Oracle for the tiled Cholesky path: TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of
``bench.py`` may import this package. It shares no code with the CUDA library and never
imports it.

* ``cholesky`` / ``forward_solve`` / ``backward_solve`` / ``solve`` wrap the plain C
  definitions in ``oracle.c`` (binary64, unblocked, no fused multiply-add).
* ``backward_error`` is the normwise (Rigal-Gaches) backward error of a computed solution,
  the quantity the accuracy target is stated in (the paper is silent on the norm; the
  infinity norm per right-hand side, maximised over columns, is the reading used here).
* ``dag`` derives the tile task graph from data access modes (Section 2, "Execution flow":
  a task becomes ready when its predecessors have completed).
* ``sched`` restates Algorithm 1 (HEFT activate) and Algorithm 2 (DADA activate) for one
  activation on identical workers.
* ``simulate`` runs the data-flow loop (Section 2) in simulated time on W identical
  workers with a given placement, so whole schedules can be checked on the CPU.
* ``lu`` is the tile LU with incremental pivoting (PLASMA DGETRF, the paper's second
  workload, Section 4.1) and its solve, kernel by kernel in program order (numpy).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_cholesky.restype = ctypes.c_int
        L.oracle_cholesky.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_long,
                                      ctypes.POINTER(ctypes.c_int)]
        for name in ("oracle_forward_solve", "oracle_backward_solve", "oracle_cholesky_solve"):
            f = getattr(L, name)
            f.restype = None
            f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_long,
                          ctypes.c_void_p, ctypes.c_long]
        L.oracle_num_threads.restype = ctypes.c_int
        L.oracle_num_threads.argtypes = []
        _LIB = L
    return _LIB


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def _fortran(a):
    return np.array(a, dtype=np.float64, order="F", copy=True)


def cholesky(A):
    """Return (F, info): F is A with its lower triangle overwritten by L (upper untouched)."""
    F = _fortran(A)
    n = F.shape[0]
    assert F.shape == (n, n)
    info = ctypes.c_int(0)
    lib().oracle_cholesky(n, F.ctypes.data, max(n, 1), ctypes.byref(info))
    return F, int(info.value)


def factor(A):
    """Lower factor L (upper triangle zeroed). Raises if A is not positive definite."""
    F, info = cholesky(A)
    if info != 0:
        raise np.linalg.LinAlgError("leading minor of order %d is not positive definite" % info)
    return np.tril(F)


def _solve_call(fn, L, B):
    L = _fortran(L)
    B = np.asarray(B, dtype=np.float64)
    vec = B.ndim == 1
    X = _fortran(B.reshape(B.shape[0], -1))
    n, nrhs = X.shape
    fn(n, nrhs, L.ctypes.data, max(n, 1), X.ctypes.data, max(n, 1))
    return X.reshape(-1) if vec else X


def forward_solve(L, B):
    return _solve_call(lib().oracle_forward_solve, L, B)


def backward_solve(L, B):
    return _solve_call(lib().oracle_backward_solve, L, B)


def solve(L, B):
    return _solve_call(lib().oracle_cholesky_solve, L, B)


def backward_error(A, X, B):
    """max over columns of ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)."""
    A = np.asarray(A, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64).reshape(A.shape[0], -1)
    B = np.asarray(B, dtype=np.float64).reshape(A.shape[0], -1)
    R = B - A @ X
    normA = np.abs(A).sum(axis=1).max() if A.size else 0.0
    num = np.abs(R).max(axis=0)
    den = normA * np.abs(X).max(axis=0) + np.abs(B).max(axis=0)
    return float((num / den).max()) if num.size else 0.0


def rel_frobenius(X, Y):
    """||X - Y||_F / ||Y||_F."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    return float(np.linalg.norm(X - Y) / np.linalg.norm(Y))


def factor_residual(A, L):
    """||A - L L^T||_F / ||A||_F for a lower factor L."""
    L = np.tril(np.asarray(L, dtype=np.float64))
    A = np.asarray(A, dtype=np.float64)
    return float(np.linalg.norm(A - L @ L.T) / np.linalg.norm(A))
