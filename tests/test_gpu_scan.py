"""Scan parity on the GPU: the CUDA path through the C ABI against the CPU
oracle.  int32 is bit-exact; float32 on integer-valued data is bit-exact
(every partial sum < 2^24); float32 on U[-1, 1] data meets the blocked
summation bound (ceil(log2 n) + P + 1) * 2^-24 * sum |x|."""
import math

import numpy as np
import pytest

import oracle
import seeded_inputs as si
from tests.gpu_util import sample_rows, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_16214_gb300 as bp
    return bp


def run_scan(bp, x, plan=None, dtype=None):
    batch, n = x.shape
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    bp.scan_batched(xd, yd, n, batch, dtype=dtype, plan=plan)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def test_config1_fixed_plan_bit_exact(bp):
    # 1024 signals x 1024 int32 in [-1000, 1000], one fixed kernel configuration
    x = si.scan_i32(1024, 1024)
    plan = bp.make_plan(bp.OP_SCAN, 1024, P=4, spb=1, pattern=bp.PATTERN_KS)
    assert np.array_equal(run_scan(bp, x, plan), oracle.scan_i32(x))


@pytest.mark.parametrize("n", [1, 2, 8, 32, 64, 256, 1024, 4096, 8192, 32768])
def test_every_plan_int32_ragged(bp, n):
    batch = 37 if n <= 8192 else 5
    x = si.full_range_int32(1000 + n, batch * n).reshape(batch, n)  # wraps often
    ref = oracle.scan_i32(x)
    plans = bp.enumerate_plans(bp.OP_SCAN, bp.I32, n)
    assert plans
    for p in plans:
        assert np.array_equal(run_scan(bp, x, p), ref), p


@pytest.mark.parametrize("n", [32, 512, 2048])
def test_every_plan_f32_integer_valued_exact(bp, n):
    x = si.scan_f32(29, n, integer_valued=True)
    ref = oracle.scan_f32(x).astype(np.float32)
    for p in bp.enumerate_plans(bp.OP_SCAN, bp.F32, n):
        assert np.array_equal(run_scan(bp, x, p), ref), p


@pytest.mark.parametrize("n", [64, 1024, 8192])
def test_every_plan_f32_uniform_bound(bp, n):
    x = si.scan_f32(17, n)
    ref = oracle.scan_f32(x)
    absum = np.cumsum(np.abs(x.astype(np.float64)), axis=1)
    for p in bp.enumerate_plans(bp.OP_SCAN, bp.F32, n):
        y = run_scan(bp, x, p).astype(np.float64)
        bound = (math.ceil(math.log2(n)) + p.P + 1) * 2.0 ** -24 * absum
        assert np.all(np.abs(y - ref) <= bound), p


def test_wraparound_and_in_place(bp):
    x = np.array([[2**31 - 1, 1, 5, -7] * 8], dtype=np.int32)
    ref = oracle.scan_i32(x)
    xd = to_dev(x)
    bp.scan_batched(xd, xd, 32, 1)
    torch.cuda.synchronize()
    assert np.array_equal(xd.cpu().numpy(), ref)
    assert xd.cpu().numpy()[0, 1] == -(2**31)


def test_default_plan_full_size_sampled(bp):
    # 2^26 elements at n = 1024 (the paper's 2^26/N batching), default plan
    n, batch = 1024, (1 << 26) // 1024
    x = si.scan_i32(batch, n, stream=3)
    y = run_scan(bp, x)
    rows = sample_rows(batch)
    assert np.array_equal(y[rows], oracle.scan_i32(x[rows]))


def test_argument_errors(bp):
    x = torch.zeros(64, dtype=torch.int32, device="cuda")
    # above 2^15 the library refuses before any launch (raw pointers: the
    # binding's tensor-size check is not involved); every smaller n is valid
    assert bp.lib.bplg_scan_batched(bp.I32, x.data_ptr(), x.data_ptr(), (1 << 15) + 1, 1, None, None) == \
        bp.ERR_UNSUPPORTED_SIZE
    with pytest.raises(bp.BplgError) as e:
        bp.scan_batched(x.data_ptr() + 4, x, 16, 1, dtype=bp.I32)
    assert e.value.code == bp.ERR_INVALID_ARG
    bad = bp.make_plan(bp.OP_SCAN, 64, P=4, spb=3)  # L = 48 is not a warp multiple
    with pytest.raises(bp.BplgError) as e:
        bp.scan_batched(x, x, 64, 1, plan=bad)
    assert e.value.code == bp.ERR_INVALID_PLAN
