"""Seeded synthetic workloads shared by the CUDA path's tests, the oracle's
tests and the benchmark.

This module holds no arithmetic of the method (no scan, no FFT, no
tridiagonal elimination).  It only draws numbers.  The generator is
SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), evaluated in counter form: the i-th output of a
stream with seed ``s`` is ``mix(s + (i + 1) * GOLDEN)``, so any element of any
stream can be drawn independently and the sequences are identical on every
machine.

Workload shapes and value distributions follow the paper's experimental
set-up (Section VI: batches of 2^26/N problems of power-of-two size N, single
precision) and the five synthetic configurations this library is measured on:

* scan:    int32 uniform on [-1000, 1000], or float32 uniform on [-1, 1];
* FFT:     complex64 with real and imaginary parts uniform on [-1, 1];
* tridiag: a, c uniform on [-1, 1]; b = |a| + |c| + U[1, 2] (strict row
  diagonal dominance with margin >= 1); x_true uniform on [-1, 1];
  d = A x_true evaluated in float64 and rounded once to float32.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# one 64-bit base seed per synthetic configuration (scan, FFT, tridiag,
# uneven batch, precision variant)
CONFIG_SEEDS = {
    "scan": 0xB9160000,
    "fft": 0xB9160001,
    "tridiag": 0xB9160002,
    "uneven": 0xB9160003,
    "precision": 0xB9160004,
}


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of the SplitMix64 stream ``seed``."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def stream_seed(base: int, stream: int) -> int:
    """Seed of sub-stream ``stream`` (one per array) of a configuration."""
    return int(splitmix64(base, 1, start=stream)[0])


def uniform01_f32(seed: int, count: int) -> np.ndarray:
    """float32 uniform on [0, 1) with 24 random bits (every value exact)."""
    z = splitmix64(seed, count)
    return ((z >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)).astype(np.float32)


def uniform_pm1_f32(seed: int, count: int) -> np.ndarray:
    """float32 uniform on [-1, 1) (exact: 2u - 1 with u on a 2^-24 grid)."""
    u = uniform01_f32(seed, count).astype(np.float64)
    return (2.0 * u - 1.0).astype(np.float32)


def uniform_int32(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """int32 uniform on [lo, hi] (modulo reduction of the high 32 bits)."""
    z = splitmix64(seed, count) >> np.uint64(32)
    span = np.uint64(hi - lo + 1)
    return ((z % span).astype(np.int64) + lo).astype(np.int32)


def full_range_int32(seed: int, count: int) -> np.ndarray:
    """int32 with all 32 bits random (exercises wrap-around)."""
    z = splitmix64(seed, count) >> np.uint64(32)
    return z.astype(np.uint32).view(np.int32)


# --------------------------------------------------------------------------
# configuration generators
# --------------------------------------------------------------------------

def scan_i32(batch: int, n: int, seed: int = CONFIG_SEEDS["scan"], stream: int = 0) -> np.ndarray:
    """[batch][n] int32 uniform on [-1000, 1000]."""
    s = stream_seed(seed, stream)
    return uniform_int32(s, batch * n, -1000, 1000).reshape(batch, n)


def scan_f32(batch: int, n: int, seed: int = CONFIG_SEEDS["scan"], stream: int = 1,
             integer_valued: bool = False) -> np.ndarray:
    """[batch][n] float32: uniform on [-1, 1), or integers in [-1000, 1000]
    (every partial sum then stays below 2^24, so any summation order is exact)."""
    s = stream_seed(seed, stream)
    if integer_valued:
        return uniform_int32(s, batch * n, -1000, 1000).astype(np.float32).reshape(batch, n)
    return uniform_pm1_f32(s, batch * n).reshape(batch, n)


def fft_c64(batch: int, n: int, seed: int = CONFIG_SEEDS["fft"], stream: int = 0) -> np.ndarray:
    """[batch][n] complex64, real and imaginary parts uniform on [-1, 1)."""
    s = stream_seed(seed, stream)
    v = uniform_pm1_f32(s, 2 * batch * n).reshape(batch, n, 2)
    return v.view(np.complex64).reshape(batch, n)


def tridiag_f32(batch: int, n: int, seed: int = CONFIG_SEEDS["tridiag"], stream: int = 0):
    """Diagonally dominant batched tridiagonal systems in SoA layout.

    Returns (a, b, c, d, x_true), each [batch][n]; a[:, 0] = c[:, n-1] = 0.
    """
    base = stream_seed(seed, stream)
    m = batch * n
    a = uniform_pm1_f32(stream_seed(base, 0), m).reshape(batch, n)
    c = uniform_pm1_f32(stream_seed(base, 1), m).reshape(batch, n)
    u = (1.0 + uniform01_f32(stream_seed(base, 2), m).astype(np.float64)).astype(np.float32).reshape(batch, n)
    x_true = uniform_pm1_f32(stream_seed(base, 3), m).reshape(batch, n)
    a[:, 0] = 0.0
    c[:, n - 1] = 0.0
    b = (np.abs(a) + np.abs(c) + u).astype(np.float32)
    xt = x_true.astype(np.float64)
    d64 = b.astype(np.float64) * xt
    d64[:, 1:] += a[:, 1:].astype(np.float64) * xt[:, :-1]
    d64[:, :-1] += c[:, :-1].astype(np.float64) * xt[:, 1:]
    d = d64.astype(np.float32)
    return a, b, c, d, x_true


def uneven_sizes(count: int, seed: int, lo_exp: int = 5, hi_exp: int = 13) -> np.ndarray:
    """Power-of-two sizes 2^e, e uniform on the integers lo_exp..hi_exp."""
    z = splitmix64(seed, count) >> np.uint64(32)
    e = (z % np.uint64(hi_exp - lo_exp + 1)).astype(np.int64) + lo_exp
    return (np.int64(1) << e).astype(np.int64)
