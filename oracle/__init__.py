"""CPU oracle for the batched scan, FFT and tridiagonal solver.

Test infrastructure only: the test suite, the smoke check and the
benchmark's CPU-baseline leg are the only callers.  The library never imports
this package and this package never imports the library.

The arithmetic lives in ``oracle.c`` (plain C, float64) and, for the tuners,
in ``tuning.py`` (plain Python).  ``build()`` compiles ``oracle.c`` with gcc
into ``oracle/_build/liboracle.so``; the wrappers below only marshal numpy
arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc -O2, portable flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-D_GNU_SOURCE",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.oracle_scan_i32.argtypes = [P, P, I64, I64]
        lib.oracle_scan_i32.restype = None
        lib.oracle_scan_f32.argtypes = [P, P, I64, I64]
        lib.oracle_scan_f32.restype = None
        lib.oracle_fft_f64.argtypes = [P, P, I64, I64, ctypes.c_int]
        lib.oracle_fft_f64.restype = ctypes.c_int
        lib.oracle_dft_f64.argtypes = [P, P, I64, I64, ctypes.c_int]
        lib.oracle_dft_f64.restype = None
        lib.oracle_thomas_f64.argtypes = [P, P, P, P, P, I64, I64]
        lib.oracle_thomas_f64.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def scan_i32(x: np.ndarray) -> np.ndarray:
    """Inclusive int32 scan along the last axis, wrapping mod 2^32."""
    x = np.ascontiguousarray(x, dtype=np.int32)
    n = x.shape[-1]
    y = np.empty_like(x)
    _load().oracle_scan_i32(_ptr(x), _ptr(y), n, x.size // max(n, 1))
    return y


def scan_f32(x: np.ndarray) -> np.ndarray:
    """Inclusive scan of float32 data accumulated in float64 (float64 out)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    n = x.shape[-1]
    y = np.empty(x.shape, dtype=np.float64)
    _load().oracle_scan_f32(_ptr(x), _ptr(y), n, x.size // max(n, 1))
    return y


def _as_interleaved(x: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.complex128))


def fft(x: np.ndarray, direction: int = -1) -> np.ndarray:
    """Batched DFT along the last axis (power-of-two length), float64.

    direction -1: forward, exp(-2 pi i jk/N); +1: inverse, unnormalised."""
    xc = _as_interleaved(x)
    n = xc.shape[-1]
    out = np.empty_like(xc)
    rc = _load().oracle_fft_f64(_ptr(xc), _ptr(out), n, xc.size // max(n, 1), int(direction))
    if rc != 0:
        raise ValueError("oracle fft: length must be a power of two")
    return out


def dft(x: np.ndarray, direction: int = -1) -> np.ndarray:
    """Batched O(N^2) DFT along the last axis (any length), long double sums."""
    xc = _as_interleaved(x)
    n = xc.shape[-1]
    out = np.empty_like(xc)
    _load().oracle_dft_f64(_ptr(xc), _ptr(out), n, xc.size // max(n, 1), int(direction))
    return out


def thomas(a, b, c, d) -> np.ndarray:
    """Batched tridiagonal solve in float64 of float32 SoA systems [batch][n]."""
    arrs = [np.ascontiguousarray(v, dtype=np.float32) for v in (a, b, c, d)]
    n = arrs[1].shape[-1]
    x = np.empty(arrs[1].shape, dtype=np.float64)
    rc = _load().oracle_thomas_f64(*[_ptr(v) for v in arrs], _ptr(x), n, arrs[1].size // max(n, 1))
    if rc != 0:
        raise ValueError("oracle thomas: bad arguments")
    return x
