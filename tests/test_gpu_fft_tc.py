"""Tensor-core FFT (radix-16 stages as split hi/lo BF16 or FP16 MMA with
float32 accumulation) against the float64 oracle: relative L2 error per
signal <= 1e-5 * log2 N, forward and inverse, every plan (the tcgen05
kernels, io 0, and the mma.sync kernels, io 1), both precisions."""
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


def run(bp, z, direction, prec, plan=None):
    batch, n = z.shape
    zd = c64_to_dev(z)
    out = torch.empty_like(zd)
    bp.fft_tc_batched(zd, out, n, batch, direction, precision=prec, plan=plan)
    torch.cuda.synchronize()
    return c64_from_dev(out)


@pytest.mark.parametrize("n", [512, 1024, 2048, 4096, 8192, 16384])
@pytest.mark.parametrize("prec", [0, 1])
def test_every_plan(bp, n, prec):
    batch = 5
    z = si.fft_c64(batch, n, stream=600 + n)
    refs = {d: oracle.fft(z, d) for d in (-1, 1)}
    plans = bp.enumerate_plans(bp.OP_FFT_TC, bp.F32, n)
    assert plans
    # the tcgen05 kernels (io 0) are in the space from n = 1024 on
    assert any(p.io == 0 for p in plans) == (n >= 1024)
    for p in plans:
        for d in (-1, 1):
            err = fft_rel_err(run(bp, z, d, prec, p), refs[d]).max()
            assert err <= 1e-5 * math.log2(n), (p, d, prec, err)


@pytest.mark.parametrize("n", [1024, 4096, 16384])
def test_precision_configuration_sampled(bp, n):
    # batch = 2^26 / N signals, default plan, both precisions
    batch = (1 << 26) // n
    z = si.fft_c64(batch, n, seed=si.CONFIG_SEEDS["precision"], stream=n)
    rows = sample_rows(batch, k=24)
    ref = oracle.fft(z[rows], -1)
    for prec in (0, 1):
        X = run(bp, z, -1, prec)
        assert fft_rel_err(X[rows], ref).max() <= 1e-5 * math.log2(n)


def test_tcgen05_plans_leave_no_device_error(bp):
    n, batch = 4096, 7
    z = si.fft_c64(batch, n, stream=611)
    ref = oracle.fft(z, -1)
    for p in bp.enumerate_plans(bp.OP_FFT_TC, bp.F32, n):
        if p.io == 0:
            assert fft_rel_err(run(bp, z, -1, 1, p), ref).max() <= 1e-5 * math.log2(n), p
    assert bp.device_status() == 0


def test_argument_errors(bp):
    z = torch.zeros(2 * 1024, dtype=torch.float32, device="cuda")
    with pytest.raises(bp.BplgError) as e:
        bp.fft_tc_batched(z, z, 256, 1)
    assert e.value.code == bp.ERR_UNSUPPORTED_SIZE
    with pytest.raises(bp.BplgError) as e:
        bp.fft_tc_batched(z, z, 1024, 1, precision=7)
    assert e.value.code == bp.ERR_INVALID_ARG


def _gemm_plan(bp, n):
    plans = [p for p in bp.enumerate_plans(bp.OP_FFT_TC, bp.F32, n) if p.io == 2]
    assert len(plans) == 1, plans
    return plans[0]


@pytest.mark.parametrize("n,batch", [(4096, 613), (16384, 311)])
@pytest.mark.parametrize("prec", [0, 1])
def test_two_gemm_pass_kernel_over_many_tiles(bp, n, batch, prec):
    """The two-GEMM-pass kernel (io 2) with more tiles than persistent blocks
    and, at n = 4096, an odd batch (a last tile of one signal): sampled
    signals against the oracle, both directions, and no device error."""
    plan = _gemm_plan(bp, n)
    assert plan.L == 512
    z = si.fft_c64(batch, n, stream=620 + n)
    rows = np.unique(np.concatenate([sample_rows(batch, k=24), [batch - 1]]))
    for d in (-1, 1):
        X = run(bp, z, d, prec, plan)
        err = fft_rel_err(X[rows], oracle.fft(z[rows], d)).max()
        assert err <= 1e-5 * math.log2(n), (d, prec, err)
    assert bp.device_status() == 0


@pytest.mark.parametrize("n", [4096, 16384])
def test_two_gemm_pass_kernel_in_place(bp, n):
    plan = _gemm_plan(bp, n)
    batch = 9
    z = si.fft_c64(batch, n, stream=640 + n)
    buf = c64_to_dev(z)
    bp.fft_tc_batched(buf, buf, n, batch, -1, precision=1, plan=plan)
    torch.cuda.synchronize()
    assert fft_rel_err(c64_from_dev(buf), oracle.fft(z, -1)).max() <= 1e-5 * math.log2(n)


@pytest.mark.parametrize("n", [4096, 16384])
def test_two_gemm_pass_kernel_at_the_precision_configuration(bp, n):
    """io 2 at the precision configuration's full size (2^26 / N signals),
    both splits and directions, checked on sampled signals; it is also the
    cost model's default tensor-core plan at these sizes (measured faster
    than the radix-16 stages there)."""
    plan = _gemm_plan(bp, n)
    batch = (1 << 26) // n
    z = si.fft_c64(batch, n, seed=si.CONFIG_SEEDS["precision"], stream=n)
    rows = np.unique(np.concatenate([sample_rows(batch, k=16), [0, batch - 1]]))
    for d in (-1, 1):
        ref = oracle.fft(z[rows], d)
        for prec in (0, 1):
            X = run(bp, z, d, prec, plan)
            err = fft_rel_err(X[rows], ref).max()
            assert err <= 1e-5 * math.log2(n), (d, prec, err)
    assert bp.device_status() == 0
    assert bp.query_plan(bp.OP_FFT_TC, bp.F32, n, batch).io == 2
