"""Uneven-size batches in one graph launch, against the CPU oracle.

Scans (int32 and float32), FFTs (forward and inverse) and tridiagonal systems
with sizes 2^e, e uniform on {5..13}, each in its own buffers, are prepared
once and run with one graph launch per call; every item is compared with the
oracle at the tolerances of the batched tests (int32 scan bit-exact), and two
launches must give identical bits."""
import math

import numpy as np
import pytest

import oracle
import seeded_inputs as si
from tests.gpu_util import c64_from_dev, c64_to_dev, fft_rel_err, to_dev, tri_rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_16214_gb300 as bp
    return bp


def make_items(bp, count, seed):
    sizes = si.uneven_sizes(3 * count, seed)
    items, host = [], []
    for k in range(count):
        n = int(sizes[k])
        if k % 2 == 0:
            x = si.scan_i32(1, n, seed=seed, stream=10 * k + 1)
            dt = bp.I32
        else:
            x = si.scan_f32(1, n, seed=seed, stream=10 * k + 1, integer_valued=True)
            dt = bp.F32
        xd = to_dev(x)
        items.append({"op": bp.OP_SCAN, "n": n, "dtype": dt, "in": [xd], "out": torch.empty_like(xd)})
        host.append(("scan", dt, x))
    for k in range(count):
        n = int(sizes[count + k])
        z = si.fft_c64(1, n, seed=seed, stream=10 * k + 2)
        zd = c64_to_dev(z)
        d = -1 if k % 3 else 1
        items.append({"op": bp.OP_FFT, "n": n, "dir": d, "in": [zd], "out": torch.empty_like(zd)})
        host.append(("fft", d, z))
    for k in range(count):
        n = int(sizes[2 * count + k])
        a, b, c, d, _ = si.tridiag_f32(1, n, seed=seed, stream=10 * k + 3)
        ts = [to_dev(v) for v in (a, b, c, d)]
        items.append({"op": bp.OP_TRIDIAG, "n": n, "in": ts, "out": torch.empty_like(ts[0])})
        host.append(("tri", 0, (a, b, c, d)))
    return items, host


def check(items, host, which):
    for k in which:
        kind, arg, x = host[k]
        out = items[k]["out"]
        if kind == "scan":
            got = out.cpu().numpy()
            ref = oracle.scan_i32(x) if arg == 0 else oracle.scan_f32(x).astype(np.float32)
            assert np.array_equal(got, ref), (k, items[k]["n"])
        elif kind == "fft":
            n = items[k]["n"]
            err = fft_rel_err(c64_from_dev(out), oracle.fft(x, arg)).max()
            assert err <= 1e-5 * math.log2(n), (k, n, err)
        else:
            ref = oracle.thomas(*x)
            assert tri_rel_err(out.cpu().numpy(), ref).max() <= 1e-4, (k, items[k]["n"])


def test_small_mixed_batch_two_launches(bp):
    items, host = make_items(bp, 48, seed=si.CONFIG_SEEDS["uneven"])
    ub = bp.UnevenBatch(items)
    assert all(u > 0 for u in ub.units())
    ub.launch()
    torch.cuda.synchronize()
    check(items, host, range(len(items)))
    first = [it["out"].clone() for it in items]
    for it in items:
        it["out"].fill_(0)
    ub.launch()
    torch.cuda.synchronize()
    for a, b in zip(first, (it["out"] for it in items)):
        assert torch.equal(a, b)
    ub.close()


def test_full_uneven_configuration_sampled(bp):
    # 4096 scans + 4096 FFTs + 4096 tridiagonal systems, one graph launch
    count = 4096
    items, host = make_items(bp, count, seed=si.CONFIG_SEEDS["uneven"] + 1)
    ub = bp.UnevenBatch(items)
    ub.launch()
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    which = sorted(set(rng.integers(0, 3 * count, size=192).tolist()) | {0, count, 2 * count, 3 * count - 1})
    check(items, host, which)
    ub.close()
    assert bp.device_status() == 0


def test_rejects_bad_items(bp):
    v = torch.zeros(64, dtype=torch.int32, device="cuda")
    with pytest.raises(bp.BplgError) as e:
        bp.UnevenBatch([{"op": bp.OP_SCAN, "n": 16, "in": [v], "out": v}])
    assert e.value.code == bp.ERR_UNSUPPORTED_SIZE
    with pytest.raises(bp.BplgError) as e:
        bp.UnevenBatch([{"op": bp.OP_FFT, "n": 64, "dir": 0, "in": [v], "out": v}])
    assert e.value.code == bp.ERR_INVALID_ARG
