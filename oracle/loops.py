"""ctypes wrapper over ``oracle/liboracle.so`` (built from ``oracle/loops.c``).

Test infrastructure only; see the package docstring.  ``build()`` compiles
the library with gcc (-O2 -ffp-contract=off -fopenmp) when it is missing or
older than its source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "loops.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_vp = ctypes.c_void_p


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.or_num_threads.restype = ctypes.c_int
        L.or_set_threads.argtypes = [ctypes.c_int]
        L.or_daxpy.argtypes = [_i64, _dbl, _vp, _vp]
        L.or_daxpy_fma.argtypes = [_i64, _dbl, _vp, _vp]
        L.or_jacobi7_sweep.argtypes = [_i64, _vp, _vp]
        L.or_jacobi7.argtypes = [_i64, ctypes.c_int, _vp, _vp, _vp]
        L.or_heat7.argtypes = [_i64, ctypes.c_int, _dbl, _vp, _vp, _vp]
        L.or_spmv.argtypes = [_i64, _vp, _vp, _vp, _vp, _vp]
        L.or_spmv_rows.argtypes = [_i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.or_csr_row_stats.argtypes = [_i64, _vp, _vp]
        L.or_nbody.argtypes = [_i64, _vp, _dbl, _vp]
        L.or_nbody_rows.argtypes = [_i64, _vp, _dbl, _i64, _vp, _vp]
        L.or_nbody_batched.argtypes = [_i64, _vp, _vp, _dbl, _vp]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_vp)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def num_threads() -> int:
    return lib().or_num_threads()


def set_threads(t: int) -> None:
    lib().or_set_threads(int(t))


def daxpy(a: float, x, y, fma: bool = False) -> np.ndarray:
    """Return a*x + y (float64); inputs are not modified."""
    x = _c(x, np.float64)
    out = np.array(y, dtype=np.float64, copy=True)
    (lib().or_daxpy_fma if fma else lib().or_daxpy)(x.size, float(a), _p(x), _p(out))
    return out


def jacobi7(u0, sweeps: int) -> np.ndarray:
    """``sweeps`` 7-point Jacobi sweeps of the (N, N, N) grid u0."""
    u0 = _c(u0, np.float64)
    N = u0.shape[0]
    assert u0.shape == (N, N, N)
    out = np.empty_like(u0)
    work = np.empty_like(u0)
    lib().or_jacobi7(N, int(sweeps), _p(u0), _p(out), _p(work))
    return out


def heat7(u0, steps: int, alpha: float) -> np.ndarray:
    """``steps`` explicit heat steps u + alpha (sum of the 6 neighbours - 6 u)
    of the (N, N, N) grid u0 (zero Dirichlet ghosts)."""
    u0 = _c(u0, np.float64)
    N = u0.shape[0]
    assert u0.shape == (N, N, N)
    out = np.empty_like(u0)
    work = np.empty_like(u0)
    lib().or_heat7(N, int(steps), float(alpha), _p(u0), _p(out), _p(work))
    return out


def spmv(rowptr, col, val, x) -> np.ndarray:
    rowptr = _c(rowptr, np.int32)
    col = _c(col, np.int32)
    val = _c(val, np.float64)
    x = _c(x, np.float64)
    rows = rowptr.size - 1
    y = np.empty(rows, dtype=np.float64)
    lib().or_spmv(rows, _p(rowptr), _p(col), _p(val), _p(x), _p(y))
    return y


def spmv_rows(rowptr, col, val, x, which):
    """Return (y[which], sum_k |val_k x_col_k| for those rows)."""
    rowptr = _c(rowptr, np.int32)
    col = _c(col, np.int32)
    val = _c(val, np.float64)
    x = _c(x, np.float64)
    which = _c(which, np.int64)
    y = np.empty(which.size, dtype=np.float64)
    a = np.empty(which.size, dtype=np.float64)
    lib().or_spmv_rows(which.size, _p(which), _p(rowptr), _p(col), _p(val), _p(x), _p(y), _p(a))
    return y, a


def csr_row_stats(rowptr) -> np.ndarray:
    """(rows, nnz, mean, variance, max) of the row lengths, float64."""
    rowptr = _c(rowptr, np.int32)
    out = np.empty(5, dtype=np.float64)
    lib().or_csr_row_stats(rowptr.size - 1, _p(rowptr), _p(out))
    return out


def nbody(p4, eps: float = 1e-2) -> np.ndarray:
    """(N, 3) float64 accelerations of the float32 (N, 4) bodies."""
    p4 = _c(p4, np.float32)
    N = p4.shape[0]
    acc = np.empty((N, 3), dtype=np.float64)
    lib().or_nbody(N, _p(p4), float(eps), _p(acc))
    return acc


def nbody_rows(p4, which, eps: float = 1e-2) -> np.ndarray:
    p4 = _c(p4, np.float32)
    which = _c(which, np.int64)
    acc = np.empty((which.size, 3), dtype=np.float64)
    lib().or_nbody_rows(p4.shape[0], _p(p4), float(eps), which.size, _p(which), _p(acc))
    return acc


def nbody_batched(p4, offs, eps: float = 1e-2) -> np.ndarray:
    p4 = _c(p4, np.float32)
    offs = _c(offs, np.int32)
    acc = np.empty((p4.shape[0], 3), dtype=np.float64)
    lib().or_nbody_batched(offs.size - 1, _p(offs), _p(p4), float(eps), _p(acc))
    return acc
