"""Lengths that are not powers of two: the scan and the Wang-Mou tridiagonal
solver run the plan of the next power of two with identity padding, the FFT
runs a mixed-radix Stockham kernel for 2^a 3^b 5^c up to 12288 and
Bluestein's chirp identity over power-of-two FFTs otherwise.  Parity against the
oracle (scan bit-exact for int32, the float64 Thomas solution <= 1e-4, the
O(N^2) DFT <= 1e-5 ceil(log2 N)), closed forms at sizes the O(N^2) oracle
cannot reach, every plan of the padded size, and nothing written past n."""
import math

import numpy as np
import pytest

import oracle
import seeded_inputs as si
from tests.gpu_util import c64_from_dev, c64_to_dev, fft_rel_err, to_dev, tri_rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SENTINEL = 12345


@pytest.fixture(scope="module")
def bp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_16214_gb300 as bp
    return bp


def next_pow2(n):
    return 1 << max(0, (n - 1).bit_length())


# ------------------------------------------------------------------ scan ----

def run_scan(bp, x, plan=None, guard=64):
    batch, n = x.shape
    xin = to_dev(x.reshape(-1))
    out = torch.full((batch * n + guard,), SENTINEL, dtype=xin.dtype, device="cuda")
    bp.scan_batched(xin, out, n, batch, dtype=bp.I32 if x.dtype == np.int32 else bp.F32, plan=plan)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert np.all(o[batch * n:] == SENTINEL), "written past the last row"
    return o[:batch * n].reshape(batch, n)


@pytest.mark.parametrize("n", [1, 3, 5, 31, 33, 100, 1000, 4097, 32767])
def test_scan_i32_every_plan_bit_exact(bp, n):
    batch = 7
    x = si.scan_i32(batch, n, stream=500 + n)
    ref = oracle.scan_i32(x)
    plans = bp.enumerate_plans(bp.OP_SCAN, bp.I32, next_pow2(n)) if n > 1 else [None]
    step = max(1, len(plans) // 12)
    for p in plans[::step] + [None]:
        assert np.array_equal(run_scan(bp, x, p), ref), p


@pytest.mark.parametrize("n", [3, 100, 1000, 5000])
def test_scan_f32_padded(bp, n):
    batch = 5
    x = si.scan_f32(batch, n, stream=600 + n, integer_valued=True)
    assert np.array_equal(run_scan(bp, x).astype(np.float64), oracle.scan_f32(x))


def test_scan_plan_for_another_length_rejected(bp):
    n, batch = 100, 3
    x = si.scan_i32(batch, n, stream=7)
    with pytest.raises(bp.BplgError):
        run_scan(bp, x, bp.make_plan(bp.OP_SCAN, 256, 4, 1))  # made for 256, not 128


# --------------------------------------------------------------- tridiag ----

def run_tri(bp, sysm, plan=None, guard=64):
    a, b, c, d = sysm[:4]
    batch, n = b.shape
    ts = [to_dev(v.reshape(-1)) for v in (a, b, c, d)]
    x = torch.full((batch * n + guard,), float(SENTINEL), dtype=torch.float32, device="cuda")
    bp.tridiag_batched(*ts, x, n, batch, plan=plan)
    torch.cuda.synchronize()
    o = x.cpu().numpy()
    assert np.all(o[batch * n:] == SENTINEL), "written past the last row"
    return o[:batch * n].reshape(batch, n)


@pytest.mark.parametrize("n", [3, 5, 17, 100, 1000, 3000, 5000])
def test_tridiag_every_wm_plan(bp, n):
    batch = 9 if n <= 1000 else 3
    a, b, c, d, _ = si.tridiag_f32(batch, n, stream=700 + n)
    c[:, -1] = np.nan  # never read
    ref = oracle.thomas(a, b, c, d)
    for p in bp.enumerate_plans(bp.OP_TRIDIAG_WM, bp.F32, next_pow2(n)) + [None]:
        x = run_tri(bp, (a, b, c, d), p)
        assert np.all(np.isfinite(x)) and tri_rel_err(x, ref).max() <= 1e-4, p


def test_tridiag_cr_plan_needs_power_of_two(bp):
    n, batch = 100, 2
    sysm = si.tridiag_f32(batch, n, stream=8)
    with pytest.raises(bp.BplgError):
        run_tri(bp, sysm, bp.make_plan(bp.OP_TRIDIAG, 128, 2, 1, cr_switch=32, shuffle=1))


# ------------------------------------------------------------------- FFT ----

def tol(n):
    return 1e-5 * math.ceil(math.log2(n))


def run_fft(bp, x, direction, plan=None, guard=16):
    batch, n = x.shape
    xin = c64_to_dev(x.reshape(-1))
    out = torch.full((2 * (batch * n + guard),), float(SENTINEL), dtype=torch.float32, device="cuda")
    bp.fft_batched(xin, out, n, batch, direction, plan=plan)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert np.all(o[2 * batch * n:] == SENTINEL), "written past the last row"
    return o[:2 * batch * n].view(np.complex64).reshape(batch, n)


# lengths with a prime factor above 5: Bluestein (fused kernel for M = 32 ..
# 8192, i.e. n = 17 .. 4096; three launches below and above)
@pytest.mark.parametrize("n", [7, 14, 77, 1001, 4095])
def test_fft_bluestein_vs_dft(bp, n):
    batch = 6 if n <= 1001 else 2
    x = si.fft_c64(batch, n, stream=800 + n)
    for direction in (-1, 1):
        X = run_fft(bp, x, direction)
        ref = oracle.dft(x, direction)
        assert fft_rel_err(X, ref).max() <= tol(n), (n, direction)


# 2^a 3^b 5^c (not a power of two, at most 12288): the mixed-radix Stockham
# kernels (one per length, radices 2 .. 16); small lengths several signals a
# block (ragged last block)
@pytest.mark.parametrize("n", [3, 5, 6, 9, 10, 12, 15, 20, 25, 27, 45, 60, 81, 100, 120, 125, 243, 360, 375, 625,
                               1000, 1215, 1536, 2187, 3000])
def test_fft_mixed_radix_vs_dft(bp, n):
    batch = 37 if n <= 100 else (5 if n < 1000 else 1)
    x = si.fft_c64(batch, n, stream=1800 + n)
    for direction in (-1, 1):
        X = run_fft(bp, x, direction)
        ref = oracle.dft(x, direction)
        assert fft_rel_err(X, ref).max() <= tol(n), (n, direction)


def test_fft_mixed_radix_every_length(bp):
    """Every length with a compile-time kernel (all 2^a 3^b 5^c up to 12288
    that are not powers of two), both directions.  Below 1000 points: three
    signals (a partly filled block) against the O(N^2) oracle.  From 1000 on
    (where the O(N^2) oracle would take minutes): an impulse against its
    closed form exp(dir 2 pi i j0 k / n) and a random signal against numpy's
    float64 FFT."""
    def smooth(v):
        for p in (2, 3, 5):
            while v % p == 0:
                v //= p
        return v == 1
    lengths = [n for n in range(3, 12289) if smooth(n) and n & (n - 1)]
    assert len(lengths) == 172
    for n in lengths:
        if n < 1000:
            x = si.fft_c64(3, n, stream=5000 + n)
            for direction in (-1, 1):
                X = run_fft(bp, x, direction)
                assert fft_rel_err(X, oracle.dft(x, direction)).max() <= tol(n), (n, direction)
            continue
        k = np.arange(n, dtype=np.float64)
        j0 = (7919 * n) // 9973
        imp = np.zeros((1, n), np.complex64)
        imp[0, j0] = 1
        x = si.fft_c64(1, n, stream=5000 + n)
        for direction in (-1, 1):
            X = run_fft(bp, imp, direction).astype(np.complex128)
            ref = np.exp(direction * 2j * np.pi * ((j0 * k) % n) / n)[None, :]
            assert fft_rel_err(X, ref).max() <= tol(n), (n, direction)
            Y = run_fft(bp, x, direction)
            xd = x.astype(np.complex128)
            ref = np.fft.fft(xd, axis=-1) if direction < 0 else np.fft.ifft(xd, axis=-1) * n
            assert fft_rel_err(Y, ref).max() <= tol(n), (n, direction)


@pytest.mark.parametrize("n", [3125, 6000, 10000, 12288])
def test_fft_mixed_radix_large_closed_forms(bp, n):
    """Beyond the O(N^2) oracle's reach: an impulse at j0 gives exp(-2 pi i
    j0 k / n), a tone at f gives n at bin f (both directions), and a random
    signal survives the forward-inverse round trip."""
    k = np.arange(n, dtype=np.float64)
    j0, f = 1234 % n, 777 % n
    for direction in (-1, 1):
        imp = np.zeros((3, n), np.complex64)
        imp[:, j0] = 1
        X = run_fft(bp, imp, direction).astype(np.complex128)
        ref = np.exp(direction * 2j * np.pi * ((j0 * k) % n) / n)
        assert fft_rel_err(X, np.broadcast_to(ref, X.shape)).max() <= tol(n)
        tone = np.exp(-direction * 2j * np.pi * ((f * k) % n) / n).astype(np.complex64)[None, :]
        Y = run_fft(bp, tone, direction)[0].astype(np.complex128)
        spike = np.zeros(n, np.complex128)
        spike[f] = n
        assert np.linalg.norm(Y - spike) / np.linalg.norm(spike) <= tol(n)
    x = si.fft_c64(3, n, stream=2200 + n)
    y = run_fft(bp, run_fft(bp, x, -1), +1).astype(np.complex128) / n
    assert fft_rel_err(y, x.astype(np.complex128)).max() <= 2 * tol(n)


def test_fft_mixed_radix_large_batch_sampled(bp):
    """A full-size batch (2^24 elements of n = 1000) checked on sampled signals."""
    n = 1000
    batch = (1 << 24) // n
    x = si.fft_c64(batch, n, stream=1999)
    X = run_fft(bp, x, -1)
    rows = np.unique(np.random.default_rng(4).integers(0, batch, 24))
    assert fft_rel_err(X[rows], oracle.dft(x[rows], -1)).max() <= tol(n)


@pytest.mark.parametrize("n", [375, 3000])
def test_fft_mixed_radix_round_trip_in_place(bp, n):
    batch = 5
    x = si.fft_c64(batch, n, stream=2100 + n)
    t = c64_to_dev(x.reshape(-1))
    bp.fft_batched(t, t, n, batch, -1)
    bp.fft_batched(t, t, n, batch, +1)
    torch.cuda.synchronize()
    y = c64_from_dev(t).reshape(batch, n) / n
    assert fft_rel_err(y, x.astype(np.complex128)).max() <= 2 * tol(n)


def test_fft_bluestein_round_trip_and_in_place(bp):
    n, batch = 1000, 4
    x = si.fft_c64(batch, n, stream=901)
    t = c64_to_dev(x.reshape(-1))
    bp.fft_batched(t, t, n, batch, -1)
    bp.fft_batched(t, t, n, batch, +1)
    torch.cuda.synchronize()
    y = c64_from_dev(t).reshape(batch, n) / n
    assert fft_rel_err(y, x.astype(np.complex128)).max() <= 2 * tol(n)


@pytest.mark.parametrize("n", [100003, 1 << 20 | 1, (1 << 23) - 1])
def test_fft_bluestein_large_closed_forms(bp, n):
    # an impulse at j0 gives exp(-2 pi i j0 k / n); a tone at f gives n at f
    k = np.arange(n, dtype=np.float64)
    j0, f = 12345, 777
    imp = np.zeros((1, n), np.complex64)
    imp[0, j0] = 1
    X = run_fft(bp, imp, -1)[0].astype(np.complex128)
    ref = np.exp(-2j * np.pi * ((j0 * k) % n) / n)
    assert np.linalg.norm(X - ref) / np.linalg.norm(ref) <= tol(n)
    tone = np.exp(2j * np.pi * ((f * k) % n) / n).astype(np.complex64)[None, :]
    Y = run_fft(bp, tone, -1)[0].astype(np.complex128)
    spike = np.zeros(n, np.complex128)
    spike[f] = n
    assert np.linalg.norm(Y - spike) / np.linalg.norm(spike) <= tol(n)


def test_fft_bluestein_inner_plan(bp):
    n, batch = 300, 4
    M = next_pow2(2 * n - 1)
    x = si.fft_c64(batch, n, stream=902)
    ref = oracle.dft(x, -1)
    for p in bp.enumerate_plans(bp.OP_FFT, bp.F32, M)[::7]:
        assert fft_rel_err(run_fft(bp, x, -1, p), ref).max() <= tol(n), p
    with pytest.raises(bp.BplgError):
        run_fft(bp, x, -1, bp.enumerate_plans(bp.OP_FFT, bp.F32, 2 * M)[0])  # not made for M
