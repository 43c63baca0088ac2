"""FFTs above 16384 points (two kernels: column transforms with the
exp(dir 2 pi i k1 n2 / n) twiddle, then row transforms written in natural
order) against the float64 oracle: relative L2 error per signal
<= 1e-5 * log2 N, forward and inverse, every plan at 2^15, the default plan
up to 2^22, in place, closed forms."""
import math

import numpy as np
import pytest

import oracle
import seeded_inputs as si
from tests.gpu_util import c64_from_dev, c64_to_dev, fft_rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_16214_gb300 as bp
    return bp


def run(bp, z, direction, plan=None, in_place=False):
    batch, n = z.shape
    zd = c64_to_dev(z)
    out = zd if in_place else torch.empty_like(zd)
    bp.fft_batched(zd, out, n, batch, direction, plan=plan)
    torch.cuda.synchronize()
    return c64_from_dev(out)


def test_every_plan_2_15(bp):
    n, batch = 1 << 15, 3
    z = si.fft_c64(batch, n, stream=15)
    refs = {d: oracle.fft(z, d) for d in (-1, 1)}
    plans = bp.enumerate_plans(bp.OP_FFT, bp.F32, n)
    assert plans and all(p.n1_log > 0 for p in plans)
    # every split N1 x N2 with both inner sizes in 2^6 .. 2^14 appears
    assert {p.n1_log for p in plans} == set(range(6, 10))
    for p in plans:
        for d in (-1, 1):
            err = fft_rel_err(run(bp, z, d, p), refs[d]).max()
            assert err <= 1e-5 * math.log2(n), (p, d, err)


@pytest.mark.parametrize("logn", [16, 18, 20, 22])
def test_default_plan(bp, logn):
    n = 1 << logn
    batch = 2 if logn <= 20 else 1
    z = si.fft_c64(batch, n, stream=logn)
    for d in (-1, 1):
        err = fft_rel_err(run(bp, z, d), oracle.fft(z, d)).max()
        assert err <= 1e-5 * logn, (logn, d, err)


def test_in_place_and_closed_forms(bp):
    n = 1 << 20
    z = si.fft_c64(2, 1 << 16, stream=5)
    assert fft_rel_err(run(bp, z, -1, in_place=True), oracle.fft(z, -1)).max() <= 1e-5 * 16
    imp = np.zeros((1, n), np.complex64)
    imp[0, 0] = 1
    X = run(bp, imp, -1)[0]
    assert np.max(np.abs(X - 1)) < 1e-6
    k0 = 4321
    tone = np.exp(2j * np.pi * k0 * np.arange(n) / n).astype(np.complex64)[None, :]
    X = run(bp, tone, -1)[0]
    assert abs(X[k0] - n) < 1e-4 * n
    assert np.max(np.abs(np.delete(X, k0))) < 1e-4 * n
    assert bp.device_status() == 0


def test_maximum_size(bp):
    # n = 2^24, the largest supported length: one random signal against the
    # oracle, and a tone whose transform is n at one bin
    n = 1 << 24
    z = si.fft_c64(1, n, stream=24)
    assert fft_rel_err(run(bp, z, -1), oracle.fft(z, -1)).max() <= 1e-5 * 24
    k0 = 123457
    k = np.arange(n, dtype=np.int64)
    tone = np.exp(2j * np.pi * ((k0 * k) % n) / n).astype(np.complex64)[None, :]
    X = run(bp, tone, -1)[0]
    assert abs(X[k0] - n) < 1e-4 * n
    assert np.max(np.abs(np.delete(X, k0))) < 1e-4 * n
    assert bp.device_status() == 0


def test_sizes_beyond_the_limit_are_rejected(bp):
    v = torch.zeros(16, dtype=torch.float32, device="cuda")
    # through the C ABI with raw pointers: rejected on the size, before any launch
    rc = bp.lib.bplg_fft_batched(v.data_ptr(), v.data_ptr(), 1 << 25, 1, -1, None, None)
    assert rc == bp.ERR_UNSUPPORTED_SIZE
