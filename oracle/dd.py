"""ctypes front end of the plain-C double-double GEMM oracle (dd_oracle.c).

TEST INFRASTRUCTURE ONLY (see the package docstring).  ``build()`` compiles
dd_oracle.c with gcc -O2 -ffp-contract=off -fopenmp into oracle/_build/;
nothing here calls the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dd_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = None


def lib_path() -> str:
    return os.path.join(_OUT_DIR, f"libddoracle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile the oracle (plain C; no contraction, no fast-math, OpenMP)."""
    out = lib_path()
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = out + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
               "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        i = ctypes.c_int
        lib.oracle_ddgemm.argtypes = [i, i, i, dp, dp, i, dp, dp, i, dp, dp, i]
        lib.oracle_ddgemm.restype = None
        lib.oracle_ddgemm_entries.argtypes = [i, dp, dp, i, dp, dp, i, i, ip, ip, dp, dp]
        lib.oracle_ddgemm_entries.restype = None
        for name in ("oracle_two_sum", "oracle_two_prod"):
            getattr(lib, name).argtypes = [ctypes.c_double, ctypes.c_double, dp, dp]
            getattr(lib, name).restype = None
        for name in ("oracle_dd_add", "oracle_dd_mul"):
            getattr(lib, name).argtypes = [ctypes.c_double] * 4 + [dp, dp]
            getattr(lib, name).restype = None
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return _lib().oracle_num_threads()


def ddgemm(a_hi, a_lo, b_hi, b_lo):
    """C = A B in double-double, every entry a scalar TwoProd/TwoSum loop."""
    a_hi, a_lo, b_hi, b_lo = map(_c, (a_hi, a_lo, b_hi, b_lo))
    m, k = a_hi.shape
    k2, n = b_hi.shape
    assert k == k2 and a_lo.shape == a_hi.shape and b_lo.shape == b_hi.shape
    c_hi = np.zeros((m, n))
    c_lo = np.zeros((m, n))
    if m and n:
        _lib().oracle_ddgemm(m, n, k, _p(a_hi), _p(a_lo), max(k, 1), _p(b_hi), _p(b_lo),
                             max(n, 1), _p(c_hi), _p(c_lo), max(n, 1))
    return c_hi, c_lo


def ddgemm_entries(a_hi, a_lo, b_hi, b_lo, rows, cols):
    """The same definition for chosen entries C[rows[t], cols[t]] only."""
    a_hi, a_lo, b_hi, b_lo = map(_c, (a_hi, a_lo, b_hi, b_lo))
    m, k = a_hi.shape
    n = b_hi.shape[1]
    rows = _c(rows, np.int32)
    cols = _c(cols, np.int32)
    cnt = rows.size
    out_hi = np.zeros(cnt)
    out_lo = np.zeros(cnt)
    if cnt:
        ip = ctypes.POINTER(ctypes.c_int)
        _lib().oracle_ddgemm_entries(k, _p(a_hi), _p(a_lo), max(k, 1), _p(b_hi), _p(b_lo),
                                     max(n, 1), cnt, rows.ctypes.data_as(ip),
                                     cols.ctypes.data_as(ip), _p(out_hi), _p(out_lo))
    return out_hi, out_lo


def _pair(fn, a, b):
    x = ctypes.c_double()
    y = ctypes.c_double()
    fn(a, b, ctypes.byref(x), ctypes.byref(y))
    return x.value, y.value


def two_sum(a, b):
    return _pair(_lib().oracle_two_sum, a, b)


def two_prod(a, b):
    return _pair(_lib().oracle_two_prod, a, b)


def dd_add(ah, al, bh, bl):
    x = ctypes.c_double()
    y = ctypes.c_double()
    _lib().oracle_dd_add(ah, al, bh, bl, ctypes.byref(x), ctypes.byref(y))
    return x.value, y.value


def dd_mul(ah, al, bh, bl):
    x = ctypes.c_double()
    y = ctypes.c_double()
    _lib().oracle_dd_mul(ah, al, bh, bl, ctypes.byref(x), ctypes.byref(y))
    return x.value, y.value
