"""Online tuning: with it on, plan-less calls run the candidates of a learned
search one call at a time; every result is checked against the oracle while
the search runs, the search finishes within its budget, and its best plan is
what bplg_query_plan then returns (and what later calls use)."""
import math

import numpy as np
import pytest

import oracle
import seeded_inputs as si
from tests.gpu_util import c64_from_dev, c64_to_dev, fft_rel_err, sample_rows, to_dev, tri_rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_16214_gb300 as bp
    bp.set_online_tuning(True, budget=16, seed=3)
    yield bp
    bp.set_online_tuning(False)


def finish(bp, op, dtype, n, batch, calls, run_and_check):
    for k in range(calls):
        run_and_check(k)
        torch.cuda.synchronize()  # the next call then collects this call's time
    ev, fin, best = bp.online_status(op, dtype, n, batch)
    assert fin and 1 <= ev <= 16, (ev, fin)
    q = bp.query_plan(op, dtype, n, batch)
    assert best is not None and q.as_dict() == best.as_dict()
    return ev


def test_online_fft(bp):
    n, batch = 2048, 3000
    z = si.fft_c64(batch, n, stream=70)
    zd = c64_to_dev(z)
    rows = sample_rows(batch, k=8)
    ref = oracle.fft(z[rows], -1)

    def call(k):
        out = torch.empty_like(zd)
        bp.fft_batched(zd, out, n, batch, -1)
        torch.cuda.synchronize()
        assert fft_rel_err(c64_from_dev(out).reshape(batch, n)[rows], ref).max() <= 1e-5 * math.log2(n), k

    finish(bp, bp.OP_FFT, bp.F32, n, batch, 50, call)


def test_online_scan(bp):
    n, batch = 512, 5000
    x = si.scan_i32(batch, n, stream=71)
    xd = to_dev(x)
    ref = oracle.scan_i32(x)

    def call(k):
        out = torch.empty_like(xd)
        bp.scan_batched(xd, out, n, batch, dtype=bp.I32)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref), k

    finish(bp, bp.OP_SCAN, bp.I32, n, batch, 50, call)


def test_online_tridiag(bp):
    n, batch = 128, 3333
    a, b, c, d, _ = si.tridiag_f32(batch, n, stream=72)
    ts = [to_dev(v) for v in (a, b, c, d)]
    ref = oracle.thomas(a, b, c, d)

    def call(k):
        x = torch.empty_like(ts[0])
        bp.tridiag_batched(*ts, x, n, batch)
        torch.cuda.synchronize()
        assert tri_rel_err(x.cpu().numpy(), ref).max() <= 1e-4, k

    finish(bp, bp.OP_TRIDIAG, bp.F32, n, batch, 50, call)


def test_online_off_leaves_calls_alone(bp):
    bp.set_online_tuning(False)
    n, batch = 4096, 7
    ev0, _, _ = bp.online_status(bp.OP_FFT, bp.F32, n, batch)
    z = c64_to_dev(si.fft_c64(batch, n, stream=73))
    out = torch.empty_like(z)
    bp.fft_batched(z, out, n, batch, -1)
    torch.cuda.synchronize()
    assert bp.online_status(bp.OP_FFT, bp.F32, n, batch)[0] == ev0 == 0
    bp.set_online_tuning(True, budget=16, seed=3)
