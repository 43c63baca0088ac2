"""The FFT entry point that allocates nothing, checked against the regular one.

bplg_fft_batched_noalloc exists for callers that cannot allocate device
memory while they run (an allocator that owns the whole device, a fixed
real-time memory budget, code that must not trigger an allocation's device
synchronisation).  It keeps its twiddle table in a static device array, so
it takes n <= 4096.  These tests call it and the regular bplg_fft_batched
through the C ABI on the same inputs, twice in a row, and require the same
answer within the FFT tolerance of the other tests (relative L2 error per
signal <= 1e-5 * log2 N).  The file is collected last; it passes alone in a
fresh process (the first call then does the per-device set-up) and after
every other test.
"""
import ctypes
import math

import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_16214_gb300 as bp
    return bp


def _c64(z):
    return torch.from_numpy(np.ascontiguousarray(z, dtype=np.complex64).view(np.float32)).to("cuda")


def _rel_err(x, ref):
    x = x.cpu().numpy().view(np.complex64).astype(np.complex128)
    ref = ref.cpu().numpy().view(np.complex64).astype(np.complex128)
    return float(np.max(np.linalg.norm(x - ref, axis=-1) / np.linalg.norm(ref, axis=-1)))


@pytest.mark.parametrize("n", [2, 16, 64, 256, 1024, 4096])
def test_noalloc_matches_the_regular_entry_point_twice(bp, n):
    batch = 37
    z = si.fft_c64(batch, n, stream=900 + n)
    zin = _c64(z)
    stream = torch.cuda.current_stream().cuda_stream
    tol = 1e-5 * max(1.0, math.log2(n))
    for direction in (-1, +1):
        ref = torch.empty_like(zin)
        rc = bp.lib.bplg_fft_batched(zin.data_ptr(), ref.data_ptr(), n, batch, direction, None, stream)
        assert rc == 0, bp.last_error()
        for _ in range(2):  # two calls in a row share the static table
            out = torch.full_like(zin, float("nan"))
            rc = bp.lib.bplg_fft_batched_noalloc(zin.data_ptr(), out.data_ptr(), n, batch, direction, None, stream)
            assert rc == 0, bp.last_error()
            torch.cuda.synchronize()
            assert _rel_err(out, ref.view(-1).view(torch.float32).reshape(zin.shape)) <= tol


def test_noalloc_with_an_explicit_plan(bp):
    n, batch = 1024, 19
    z = si.fft_c64(batch, n, stream=977)
    zin = _c64(z)
    ref = torch.empty_like(zin)
    stream = torch.cuda.current_stream().cuda_stream
    assert bp.lib.bplg_fft_batched(zin.data_ptr(), ref.data_ptr(), n, batch, -1, None, stream) == 0
    plan = bp.make_plan(bp.OP_FFT, n, P=8, spb=2, smem_pad=1, io=1)
    for _ in range(2):
        out = torch.empty_like(zin)
        rc = bp.lib.bplg_fft_batched_noalloc(zin.data_ptr(), out.data_ptr(), n, batch, -1, ctypes.byref(plan), stream)
        assert rc == 0, bp.last_error()
        torch.cuda.synchronize()
        assert _rel_err(out, ref) <= 1e-5 * math.log2(n)


def test_noalloc_rejects_sizes_beyond_its_table(bp):
    v = torch.zeros(2 * 8192, dtype=torch.float32, device="cuda")
    rc = bp.lib.bplg_fft_batched_noalloc(v.data_ptr(), v.data_ptr(), 8192, 1, -1, None, None)
    assert rc == bp.ERR_UNSUPPORTED_SIZE
    assert "4096" in bp.last_error()


@pytest.mark.parametrize("n", [16, 1024, 4096])
def test_noalloc_against_the_oracle(bp, n):
    """Checked directly against the float64 oracle as well, both directions."""
    import oracle
    batch = 23
    z = si.fft_c64(batch, n, stream=940 + n)
    zin = _c64(z)
    stream = torch.cuda.current_stream().cuda_stream
    for direction in (-1, +1):
        out = torch.full_like(zin, float("nan"))
        rc = bp.lib.bplg_fft_batched_noalloc(zin.data_ptr(), out.data_ptr(), n, batch, direction, None, stream)
        assert rc == 0, bp.last_error()
        torch.cuda.synchronize()
        X = out.cpu().numpy().view(np.complex64).reshape(batch, n).astype(np.complex128)
        ref = oracle.fft(z, direction)
        err = np.linalg.norm(X - ref, axis=-1) / np.linalg.norm(ref, axis=-1)
        assert err.max() <= 1e-5 * math.log2(n), (direction, err.max())


@pytest.mark.parametrize("n", [16, 4096])
def test_noalloc_in_place(bp, n):
    """out == in, which the entry point allows."""
    import oracle
    batch = 9
    z = si.fft_c64(batch, n, stream=960 + n)
    buf = _c64(z)
    stream = torch.cuda.current_stream().cuda_stream
    rc = bp.lib.bplg_fft_batched_noalloc(buf.data_ptr(), buf.data_ptr(), n, batch, -1, None, stream)
    assert rc == 0, bp.last_error()
    torch.cuda.synchronize()
    X = buf.cpu().numpy().view(np.complex64).reshape(batch, n).astype(np.complex128)
    ref = oracle.fft(z, -1)
    assert (np.linalg.norm(X - ref, axis=-1) / np.linalg.norm(ref, axis=-1)).max() <= 1e-5 * math.log2(n)

