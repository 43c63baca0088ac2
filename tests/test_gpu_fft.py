"""Stockham FFT parity on the GPU against the float64 oracle: per-signal
relative L2 error <= 1e-5 * log2 N, forward and inverse, over every valid
plan (radix, signals per block, layout, padding, io) at several sizes with a
ragged batch, plus closed forms and full-size sampled checks."""
import math

import numpy as np
import pytest

import oracle
import seeded_inputs as si
from tests.gpu_util import c64_from_dev, c64_to_dev, fft_rel_err, sample_rows

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_16214_gb300 as bp
    return bp


def tol(n):
    return 1e-5 * max(1.0, math.log2(n))


def run_fft(bp, z, direction, plan=None, in_place=False):
    batch, n = z.shape
    zd = c64_to_dev(z)
    out = zd if in_place else torch.empty_like(zd)
    bp.fft_batched(zd, out, n, batch, direction, plan=plan)
    torch.cuda.synchronize()
    return c64_from_dev(out)


@pytest.mark.parametrize("n", [2, 4, 16, 32, 64, 128, 256, 1024, 2048, 4096, 8192, 16384])
def test_every_plan_fwd_inv_ragged(bp, n):
    batch = 13 if n <= 4096 else 3
    z = si.fft_c64(batch, n, stream=n)
    ref_f = oracle.fft(z, -1)
    ref_i = oracle.fft(z, +1)
    plans = bp.enumerate_plans(bp.OP_FFT, bp.F32, n)
    assert plans
    for p in plans:
        assert fft_rel_err(run_fft(bp, z, -1, p), ref_f).max() <= tol(n), p
        assert fft_rel_err(run_fft(bp, z, +1, p), ref_i).max() <= tol(n), p


@pytest.mark.parametrize("n", [16, 512, 8192])
def test_default_plan_and_in_place(bp, n):
    z = si.fft_c64(9, n, stream=5)
    ref = oracle.fft(z, -1)
    assert fft_rel_err(run_fft(bp, z, -1), ref).max() <= tol(n)
    assert fft_rel_err(run_fft(bp, z, -1, in_place=True), ref).max() <= tol(n)


def test_closed_forms_on_gpu(bp):
    n = 256
    k = np.arange(n)
    imp = np.zeros((2, n), np.complex64)
    imp[:, 0] = 1
    assert np.allclose(run_fft(bp, imp, -1), 1.0, atol=1e-6)
    tone = np.exp(2j * np.pi * 17 * k / n).astype(np.complex64)[None, :]
    X = run_fft(bp, tone, -1)[0]
    assert abs(X[17] - n) < 1e-3 and np.max(np.abs(np.delete(X, 17))) < 1e-3
    z = si.fft_c64(4, n, stream=11)
    back = run_fft(bp, run_fft(bp, z, -1), +1) / n
    assert np.max(np.abs(back - z)) < 1e-5


@pytest.mark.parametrize("n", [16, 64, 256, 1024, 4096])
def test_full_size_default_plan_sampled(bp, n):
    # batch = 2^24 / N signals, the configuration the benchmark times
    batch = (1 << 24) // n
    z = si.fft_c64(batch, n, stream=21)
    rows = sample_rows(batch)
    for direction in (-1, +1):
        X = run_fft(bp, z, direction)
        assert fft_rel_err(X[rows], oracle.fft(z[rows], direction)).max() <= tol(n)


def test_argument_errors(bp):
    z = torch.zeros(2 * 64, dtype=torch.float32, device="cuda")
    # sizes the library rejects before any launch (raw pointers: the binding's
    # tensor-size check is not involved)
    for n in ((1 << 23) + 1, 1 << 25):  # above the Bluestein limit / above 2^24
        assert bp.lib.bplg_fft_batched(z.data_ptr(), z.data_ptr(), n, 1, -1, None, None) == bp.ERR_UNSUPPORTED_SIZE
    # a tensor too small for n x batch is refused by the binding
    with pytest.raises(ValueError):
        bp.fft_batched(z, z, 1 << 15, 1)
    with pytest.raises(bp.BplgError) as e:
        bp.fft_batched(z, z, 64, 1, direction=0)
    assert e.value.code == bp.ERR_INVALID_ARG
    bad = bp.make_plan(bp.OP_FFT, 64, P=8, spb=4, radix=4)  # P must equal the radix
    with pytest.raises(bp.BplgError) as e:
        bp.fft_batched(z, z, 64, 1, plan=bad)
    assert e.value.code == bp.ERR_INVALID_PLAN


def test_no_device_error_recorded(bp):
    # every pipelined launch above completed its bounded waits
    assert bp.device_status() == 0
