"""Oracle (test infrastructure only; never on the product path).

ctypes front end of oracle/jacobi.c: one-sided Jacobi SVD and cyclic
Jacobi Hermitian eigensolver, real and complex, column-major FP64.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        for suf in ("_d", "_z"):
            f = getattr(lib, "oracle_jacobi_svd" + suf)
            f.restype = ctypes.c_int
            f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                          ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                          ctypes.c_int, ctypes.c_int]
            g = getattr(lib, "oracle_jacobi_eig" + suf)
            g.restype = ctypes.c_int
            g.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                          ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                          ctypes.c_int, ctypes.c_int]
        _lib = lib
    return _lib


def threads() -> int:
    v = os.environ.get("ORACLE_THREADS")
    return int(v) if v else (os.cpu_count() or 1)


def _suffix(a):
    return "_z" if np.iscomplexobj(a) else "_d"


def svd_onesided(A, max_sweeps=80):
    """One-sided Jacobi SVD.  Returns (G, V, sigma, sweeps) with A V = G and
    the columns of G mutually orthogonal (G = U Sigma)."""
    lib = _load()
    dt = np.complex128 if np.iscomplexobj(A) else np.float64
    G = np.array(A, dtype=dt, order="F", copy=True)
    m, n = G.shape
    V = np.zeros((n, n), dtype=dt, order="F")
    sigma = np.zeros(n, dtype=np.float64)
    fn = getattr(lib, "oracle_jacobi_svd" + _suffix(G))
    sw = fn(m, n, G.ctypes.data, max(m, 1), V.ctypes.data, max(n, 1),
            sigma.ctypes.data, max_sweeps, threads())
    if sw < 0:
        raise RuntimeError("oracle one-sided Jacobi SVD did not converge")
    return G, V, sigma, sw


def eig_cyclic(B, max_sweeps=80):
    """Cyclic Jacobi eigendecomposition of a Hermitian B (unsorted).
    Returns (lambda, V, sweeps) with B V = V diag(lambda)."""
    lib = _load()
    dt = np.complex128 if np.iscomplexobj(B) else np.float64
    Bw = np.array(B, dtype=dt, order="F", copy=True)
    n = Bw.shape[0]
    V = np.zeros((n, n), dtype=dt, order="F")
    lam = np.zeros(n, dtype=np.float64)
    fn = getattr(lib, "oracle_jacobi_eig" + _suffix(Bw))
    sw = fn(n, Bw.ctypes.data, max(n, 1), V.ctypes.data, max(n, 1),
            lam.ctypes.data, max_sweeps, threads())
    if sw < 0:
        raise RuntimeError("oracle cyclic Jacobi eigensolver did not converge")
    return lam, V, sw
