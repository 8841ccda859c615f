"""Oracle for the multi-level 2-D DWT -- TEST INFRASTRUCTURE ONLY.

A plain, slow CPU statement of what the paper's transform computes (separable
1-D lifting of Sec. 2.2 applied to columns then rows, re-applied to LL for
each level), in FP64 for the float wavelets and exact int64 for the JPEG 2000
reversible 5/3.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the product library never does.

The C source (``dwt_oracle.c``) is compiled on first use into
``oracle/liboracle.so`` with gcc; :func:`build` does it explicitly.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

__all__ = [
    "CDF53", "CDF97", "DD137", "NORM_JPEG2000", "NORM_ZETA", "build", "lib",
    "mirror", "cdf97_constants", "lifting", "dwt1", "dwt1_int", "dwt2",
    "dwt2_int", "dwt2_int_iwahashi", "max_levels", "OracleRangeError",
]

CDF53, CDF97, DD137 = 0, 1, 2
NORM_JPEG2000, NORM_ZETA = 0, 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dwt_oracle.c")
_HDR = os.path.join(_HERE, "dwt_oracle.h")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None


class OracleRangeError(ArithmeticError):
    """An integer intermediate left the int32 range."""


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no vector intrinsics)."""
    stale = (not os.path.exists(_SO) or
             os.path.getmtime(_SO) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        l = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int64)
        l.oracle_mirror.argtypes = [ctypes.c_long, ctypes.c_long]
        l.oracle_mirror.restype = ctypes.c_long
        l.oracle_cdf97_constants.argtypes = [dp]
        l.oracle_cdf97_constants.restype = ctypes.c_double
        l.oracle_lifting.argtypes = [ctypes.c_int, dp, dp, dp, dp, dp, dp, ctypes.c_int]
        l.oracle_lifting.restype = ctypes.c_int
        l.oracle_dwt1_f64.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_long, dp, ctypes.c_long]
        l.oracle_dwt1_f64.restype = ctypes.c_int
        l.oracle_dwt1_i64.argtypes = [ctypes.c_int, ctypes.c_long, ip, ctypes.c_long]
        l.oracle_dwt1_i64.restype = ctypes.c_int
        l.oracle_dwt2_f64.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, dp, dp]
        l.oracle_dwt2_f64.restype = ctypes.c_int
        l.oracle_dwt2_i64.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ip]
        l.oracle_dwt2_i64.restype = ctypes.c_int
        l.oracle_dwt2_iwahashi_i64.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ip]
        l.oracle_dwt2_iwahashi_i64.restype = ctypes.c_int
        l.oracle_max_levels.argtypes = [ctypes.c_int, ctypes.c_int]
        l.oracle_max_levels.restype = ctypes.c_int
        _lib = l
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def mirror(i: int, n: int) -> int:
    """Whole-sample symmetric index of position ``i`` on a line of length ``n``."""
    return lib().oracle_mirror(i, n)


def cdf97_constants():
    """(alpha, beta, gamma, delta, K, residual): 9/7 lifting constants derived
    from the vanishing-moment conditions, and the unscaled low-pass DC gain."""
    out = np.zeros(5)
    res = lib().oracle_cdf97_constants(_dptr(out))
    return (*out.tolist(), res)


def lifting(wavelet: int, norm: int = NORM_JPEG2000):
    """Lifting coefficients: dict with K, pred1/pred3/upd1/upd3 (per pair) and
    the scaling of the low and high bands."""
    p1, p3, u1, u3 = (np.zeros(2) for _ in range(4))
    slo, shi = np.zeros(1), np.zeros(1)
    K = lib().oracle_lifting(wavelet, _dptr(p1), _dptr(p3), _dptr(u1), _dptr(u3), _dptr(slo), _dptr(shi), norm)
    if K < 0:
        raise ValueError("unknown wavelet")
    return dict(K=K, pred1=p1[:K].tolist(), pred3=p3[:K].tolist(), upd1=u1[:K].tolist(),
                upd3=u3[:K].tolist(), scale_lo=float(slo[0]), scale_hi=float(shi[0]))


def max_levels(w: int, h: int) -> int:
    return lib().oracle_max_levels(w, h)


def dwt1(x, wavelet: int, inverse: bool = False, norm: int = NORM_JPEG2000) -> np.ndarray:
    """1-D transform of one line; forward output = [lows | highs]."""
    a = np.ascontiguousarray(x, dtype=np.float64).copy()
    if lib().oracle_dwt1_f64(wavelet, norm, int(inverse), a.size, _dptr(a), 1) != 0:
        raise ValueError("invalid arguments")
    return a


def dwt1_int(x, inverse: bool = False) -> np.ndarray:
    a = np.ascontiguousarray(x, dtype=np.int64).copy()
    if lib().oracle_dwt1_i64(int(inverse), a.size, _iptr(a), 1) != 0:
        raise ValueError("invalid arguments")
    return a


def dwt2(x, wavelet: int, levels: int, inverse: bool = False, norm: int = NORM_JPEG2000) -> np.ndarray:
    """L-level 2-D transform of an (h, w) image in FP64, Mallat-packed."""
    a = np.ascontiguousarray(x, dtype=np.float64)
    h, w = a.shape
    out = np.empty_like(a)
    rc = lib().oracle_dwt2_f64(wavelet, norm, int(inverse), w, h, levels, _dptr(a), _dptr(out))
    if rc != 0:
        raise ValueError(f"invalid arguments (rc={rc})")
    return out


def dwt2_int(x, levels: int, inverse: bool = False) -> np.ndarray:
    """L-level reversible integer 5/3 (JPEG 2000 floor rounding), exact int64
    with an int32 range check on every intermediate."""
    a = np.ascontiguousarray(x, dtype=np.int64)
    h, w = a.shape
    out = np.empty_like(a)
    rc = lib().oracle_dwt2_i64(int(inverse), w, h, levels, _iptr(a), _iptr(out))
    if rc == -2:
        raise OracleRangeError("an intermediate left the int32 range")
    if rc != 0:
        raise ValueError(f"invalid arguments (rc={rc})")
    return out


def dwt2_int_iwahashi(x, levels: int, inverse: bool = False) -> np.ndarray:
    """L-level reversible integer non-separable lifting (the Iwahashi scheme
    of CDF 5/3 with each step's update rounded once), exact int64 with an
    int32 range check; see dwt_oracle.h for the definition."""
    a = np.ascontiguousarray(x, dtype=np.int64)
    h, w = a.shape
    out = np.empty_like(a)
    rc = lib().oracle_dwt2_iwahashi_i64(int(inverse), w, h, levels, _iptr(a), _iptr(out))
    if rc == -2:
        raise OracleRangeError("an intermediate left the int32 range")
    if rc != 0:
        raise ValueError(f"invalid arguments (rc={rc})")
    return out
