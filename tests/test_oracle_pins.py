"""Pins for the CPU oracle: each check compares it with something other than
itself -- brute force, closed forms, invariants, an independent library
routine (numpy / LAPACK), or the paper's printed tables.  No GPU needed."""
import math

import numpy as np
import pytest

import oracle
import seeded_inputs as si
from oracle import tuning as T


# ----------------------------------------------------------------- scan ----

def test_scan_i32_brute_force_small():
    x = si.scan_i32(5, 64)
    y = oracle.scan_i32(x)
    for s in range(5):
        for i in range(64):
            ref = sum(int(v) for v in x[s, : i + 1])
            ref = ((ref + 2**31) % 2**32) - 2**31
            assert y[s, i] == ref


def test_scan_i32_closed_forms():
    n = 1000
    assert np.array_equal(oracle.scan_i32(np.ones((2, n), np.int32))[0], np.arange(1, n + 1))
    e = np.zeros((1, n), np.int32)
    e[0, 137] = 5
    y = oracle.scan_i32(e)[0]
    assert np.all(y[:137] == 0) and np.all(y[137:] == 5)


def test_scan_i32_wraparound():
    x = np.array([[2**31 - 1, 1, -1, -(2**31)]], np.int32)
    y = oracle.scan_i32(x)[0]
    assert y[0] == 2**31 - 1
    assert y[1] == -(2**31)          # INT32_MAX + 1 wraps to INT32_MIN
    assert y[2] == 2**31 - 1
    assert y[3] == -1


def test_scan_i32_full_range_vs_uint64_mod():
    x = si.full_range_int32(12345, 4 * 4096).reshape(4, 4096)
    ref = (np.cumsum(x.astype(np.int64), axis=1) % 2**32).astype(np.uint32).view(np.int32)
    assert np.array_equal(oracle.scan_i32(x), ref)


def test_scan_f32_matches_exact_sums():
    x = si.scan_f32(3, 257)
    y = oracle.scan_f32(x)
    for s in range(3):
        for i in (0, 1, 100, 256):
            exact = math.fsum(float(v) for v in x[s, : i + 1])
            # sequential float64 summation: |err| <= i * 2^-53 * sum |x|
            bound = (i + 1) * 2.0**-53 * float(np.abs(x[s, : i + 1]).sum())
            assert abs(y[s, i] - exact) <= bound


def test_scan_f32_integer_valued_exact():
    x = si.scan_f32(4, 4096, integer_valued=True)
    ref = np.cumsum(x.astype(np.int64), axis=1).astype(np.float64)
    assert np.array_equal(oracle.scan_f32(x), ref)


# ------------------------------------------------------------------ FFT ----

@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 64, 256, 1024])
def test_fft_vs_numpy_and_dft(n):
    x = si.fft_c64(3, n).astype(np.complex128)
    X = oracle.fft(x, -1)
    ref = np.fft.fft(x, axis=-1)
    scale = np.linalg.norm(ref) + 1e-300
    assert np.linalg.norm(X - ref) / scale < 1e-13
    if n <= 256:
        D = oracle.dft(x, -1)
        assert np.linalg.norm(D - ref) / scale < 1e-13
        assert np.linalg.norm(X - D) / scale < 1e-13
    Xi = oracle.fft(x, +1)
    assert np.linalg.norm(Xi - n * np.fft.ifft(x, axis=-1)) / scale < 1e-13


@pytest.mark.parametrize("fn", [oracle.fft, oracle.dft])
def test_fft_closed_forms(fn):
    n = 64
    k = np.arange(n)
    imp = np.zeros((1, n), np.complex128)
    imp[0, 0] = 1
    assert np.allclose(fn(imp, -1)[0], np.ones(n), atol=1e-13)
    m = 5
    dm = np.zeros((1, n), np.complex128)
    dm[0, m] = 1
    assert np.allclose(fn(dm, -1)[0], np.exp(-2j * np.pi * m * k / n), atol=1e-13)
    assert np.allclose(fn(dm, +1)[0], np.exp(+2j * np.pi * m * k / n), atol=1e-13)
    const = np.ones((1, n), np.complex128)
    ref = np.zeros(n, np.complex128)
    ref[0] = n
    assert np.allclose(fn(const, -1)[0], ref, atol=1e-12)
    k0 = 7
    tone = np.exp(2j * np.pi * k0 * k / n)[None, :]
    ref = np.zeros(n, np.complex128)
    ref[k0] = n
    assert np.allclose(fn(tone, -1)[0], ref, atol=1e-11)


def test_fft_invariants():
    n = 512
    x = si.fft_c64(4, n).astype(np.complex128)
    X = oracle.fft(x, -1)
    # Parseval
    assert np.allclose(np.sum(np.abs(x) ** 2, axis=1), np.sum(np.abs(X) ** 2, axis=1) / n, rtol=1e-12)
    # inverse round trip: inv(fwd(x)) = N x
    assert np.allclose(oracle.fft(X, +1), n * x, atol=1e-10)
    # linearity
    y = si.fft_c64(4, n, stream=7).astype(np.complex128)
    assert np.allclose(oracle.fft(2.5 * x - 1j * y, -1), 2.5 * X - 1j * oracle.fft(y, -1), atol=1e-10)
    # real input -> Hermitian spectrum
    r = x.real.astype(np.complex128)
    R = oracle.fft(r, -1)
    assert np.allclose(R[:, 1:], np.conj(R[:, :0:-1]), atol=1e-11)


@pytest.mark.parametrize("n", [1 << 15, 1 << 18, 1 << 20])
def test_fft_large_vs_numpy(n):
    # the sizes of the two-pass large-transform path
    x = si.fft_c64(2, n, stream=31).astype(np.complex128)
    for d in (-1, 1):
        X = oracle.fft(x, d)
        ref = np.fft.fft(x, axis=-1) if d < 0 else n * np.fft.ifft(x, axis=-1)
        assert np.linalg.norm(X - ref) / np.linalg.norm(ref) < 1e-13


def test_fft_large_closed_forms():
    n = 1 << 20
    k = np.arange(n)
    m = 12345
    dm = np.zeros((1, n), np.complex128)
    dm[0, m] = 1
    assert np.allclose(oracle.fft(dm, -1)[0], np.exp(-2j * np.pi * m * k / n), atol=1e-11)
    k0 = 777
    tone = np.exp(2j * np.pi * k0 * k / n)[None, :]
    X = oracle.fft(tone, -1)[0]
    assert abs(X[k0] - n) < 1e-6 * n and np.max(np.abs(np.delete(X, k0))) < 1e-6 * n


def test_fft_rejects_non_pow2():
    with pytest.raises(ValueError):
        oracle.fft(np.zeros((1, 12), np.complex128))


# ------------------------------------------------------------- tridiag ----

def _dense(a, b, c):
    n = b.shape[0]
    A = np.diag(b.astype(np.float64))
    A += np.diag(a[1:].astype(np.float64), -1)
    A += np.diag(c[:-1].astype(np.float64), 1)
    return A


@pytest.mark.parametrize("n", [1, 2, 3, 8, 32, 64])
def test_thomas_vs_lapack(n):
    a, b, c, d, xt = si.tridiag_f32(4, n)
    x = oracle.thomas(a, b, c, d)
    for s in range(4):
        ref = np.linalg.solve(_dense(a[s], b[s], c[s]), d[s].astype(np.float64))
        assert np.max(np.abs(x[s] - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


def test_thomas_closed_forms():
    n = 16
    b = np.linspace(1, 3, n, dtype=np.float32)[None, :]
    d = np.linspace(-2, 2, n, dtype=np.float32)[None, :]
    z = np.zeros_like(b)
    assert np.allclose(oracle.thomas(z, b, z, d)[0], d[0].astype(np.float64) / b[0].astype(np.float64), rtol=0, atol=1e-15)
    # n = 2 by Cramer's rule
    a = np.array([[0.0, 0.75]], np.float32)
    bb = np.array([[2.0, 3.0]], np.float32)
    c = np.array([[-0.5, 0.0]], np.float32)
    dd = np.array([[1.0, 2.0]], np.float32)
    det = 2.0 * 3.0 - (-0.5) * 0.75
    x0 = (1.0 * 3.0 - (-0.5) * 2.0) / det
    x1 = (2.0 * 2.0 - 0.75 * 1.0) / det
    assert np.allclose(oracle.thomas(a, bb, c, dd)[0], [x0, x1], rtol=0, atol=1e-15)


def test_thomas_residual_and_known_solution():
    n = 1024
    a, b, c, d, xt = si.tridiag_f32(8, n)
    x = oracle.thomas(a, b, c, d)
    r = b.astype(np.float64) * x - d.astype(np.float64)
    r[:, 1:] += a[:, 1:].astype(np.float64) * x[:, :-1]
    r[:, :-1] += c[:, :-1].astype(np.float64) * x[:, 1:]
    normA = np.max(np.abs(a) + np.abs(b) + np.abs(c), axis=1).astype(np.float64)
    assert np.all(np.max(np.abs(r), axis=1) / (normA * np.max(np.abs(x), axis=1)) <= 1e-15)
    # x differs from x_true only through rounding d to float32: ||A^-1|| <= 1
    assert np.max(np.abs(x - xt)) <= 2.0**-24 * 4.0


def test_thomas_ignores_outside_coefficients():
    a, b, c, d, _ = si.tridiag_f32(2, 32)
    x0 = oracle.thomas(a, b, c, d)
    a2, c2 = a.copy(), c.copy()
    a2[:, 0] = np.nan
    c2[:, -1] = np.nan
    assert np.array_equal(oracle.thomas(a2, b, c2, d), x0)


# ------------------------------------------------------------- tuning ----

def test_occupancy_matches_fig2a(golden):
    for w, r, s, occ, blocks, pinned in golden("occupancy_gm20b.txt"):
        W, B = T.occupancy(T.TX1, int(w), int(r), int(s))
        if pinned == "yes":
            assert round(100 * W / 64) == int(occ) and B == int(blocks), (w, r, s)
        else:
            assert (round(100 * W / 64), B) != (int(occ), int(blocks))


def test_guideline_reproduces_fig2bcd(golden):
    for op, N, S, P, L in golden("analytic_tuples_tx1.txt"):
        assert T.paper_tuple(op, int(N)) == (int(S), int(P), int(L)), (op, N)


def test_occupancy_limits():
    # a block above the thread cap, register cap or smem cap cannot launch
    assert T.occupancy(T.TX1, 33, 32, 0) == (0, 0)
    assert T.occupancy(T.TX1, 2, 256, 0) == (0, 0)
    assert T.occupancy(T.TX1, 2, 32, 49153) == (0, 0)
    # the GB300 reserves 1 KB per block: 227 KB blocks fit once per SM
    assert T.occupancy(T.GB300, 8, 32, 232448)[1] == 1
    assert T.occupancy(T.GB300, 8, 32, 0)[1] == 8


def test_phi_closed_form():
    assert T.phi([1.0, 1.0, 1.0]) == 1.0
    assert abs(T.phi([1.0, 0.5]) - 2.0 / 3.0) < 1e-15
    assert abs(T.phi([0.9] * 7) - 0.9) < 1e-15
    assert T.phi([]) == 0.0


# ------------------------------------------- lengths that are not powers of two

@pytest.mark.parametrize("n", [3, 5, 6, 7, 12, 100, 243, 1000])
def test_dft_any_length_vs_numpy(n):
    # the O(N^2) oracle is the reference for the Bluestein path: it must hold
    # for every length, not only powers of two
    x = si.fft_c64(2, n, stream=n).astype(np.complex128)
    ref = np.fft.fft(x, axis=-1)
    scale = np.linalg.norm(ref)
    assert np.linalg.norm(oracle.dft(x, -1) - ref) / scale < 1e-13
    assert np.linalg.norm(oracle.dft(x, +1) - n * np.fft.ifft(x, axis=-1)) / scale < 1e-13


@pytest.mark.parametrize("n", [3, 35, 1000])
def test_dft_any_length_closed_forms(n):
    k = np.arange(n)
    j0, f = min(2, n - 1), min(4, n - 1)
    imp = np.zeros((1, n), np.complex128)
    imp[0, j0] = 1
    assert np.allclose(oracle.dft(imp, -1)[0], np.exp(-2j * np.pi * j0 * k / n), atol=1e-13)
    tone = np.exp(2j * np.pi * f * k / n)[None, :]
    spike = np.zeros(n, np.complex128)
    spike[f] = n
    assert np.allclose(oracle.dft(tone, -1)[0], spike, atol=1e-9 * n)


@pytest.mark.parametrize("n", [1, 3, 33, 1000])
def test_scan_and_thomas_any_length(n):
    x = si.scan_i32(3, n, stream=n)
    ref = (np.cumsum(x.astype(np.int64), axis=1) & 0xFFFFFFFF).astype(np.uint32).view(np.int32)
    assert np.array_equal(oracle.scan_i32(x), ref)
    if n >= 2:
        a, b, c, d, xt = si.tridiag_f32(2, n, stream=n)
        A = np.diag(b[0].astype(np.float64)) + np.diag(a[0, 1:].astype(np.float64), -1) + np.diag(c[0, :-1].astype(np.float64), 1)
        assert np.allclose(oracle.thomas(a, b, c, d)[0], np.linalg.solve(A, d[0].astype(np.float64)), rtol=1e-12, atol=1e-13)
