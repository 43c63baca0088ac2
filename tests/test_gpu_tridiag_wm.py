"""Wang-Mou divide-and-conquer tridiagonal solver (op BPLG_OP_TRIDIAG_WM)
against the float64 Thomas oracle on the stored float32 systems: relative
error <= 1e-4 per system over every valid plan (threads per system, systems
per block, merge radix, shuffle or shared-memory stages) with ragged
batches, the never-read outside coefficients, in-place solves, decoupled
systems, full-size batches, plan validation and the tuners."""
import numpy as np
import pytest

import oracle
import seeded_inputs as si
from tests.gpu_util import sample_rows, to_dev, tri_rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_16214_gb300 as bp
    return bp


def run_wm(bp, sysm, plan):
    a, b, c, d = sysm[:4]
    batch, n = b.shape
    ts = [to_dev(v) for v in (a, b, c, d)]
    x = torch.empty_like(ts[0])
    bp.tridiag_batched(*ts, x, n, batch, plan=plan)
    torch.cuda.synchronize()
    return x.cpu().numpy()


@pytest.mark.parametrize("n", [2, 4, 8, 16, 32, 64, 128, 256, 1024, 2048, 8192])
def test_every_plan_ragged(bp, n):
    batch = 37 if n <= 64 else (11 if n <= 2048 else 3)
    sysm = si.tridiag_f32(batch, n, stream=200 + n)
    ref = oracle.thomas(*sysm[:4])
    plans = bp.enumerate_plans(bp.OP_TRIDIAG_WM, bp.F32, n)
    assert plans
    radices = {p.radix for p in plans}
    if n >= 64:
        assert radices == {2, 4, 8}
    for p in plans:
        assert tri_rel_err(run_wm(bp, sysm, p), ref).max() <= 1e-4, p


def test_outside_coefficients_never_read(bp):
    n, batch = 256, 5
    a, b, c, d, _ = si.tridiag_f32(batch, n, stream=211)
    a[:, 0] = np.nan
    c[:, -1] = np.nan
    ref = oracle.thomas(a, b, c, d)
    for p in bp.enumerate_plans(bp.OP_TRIDIAG_WM, bp.F32, n):
        x = run_wm(bp, (a, b, c, d), p)
        assert np.all(np.isfinite(x)) and tri_rel_err(x, ref).max() <= 1e-4, p


def test_x_may_alias_d(bp):
    n, batch = 512, 7
    a, b, c, d, _ = si.tridiag_f32(batch, n, stream=212)
    ref = oracle.thomas(a, b, c, d)
    p = bp.query_plan(bp.OP_TRIDIAG_WM, bp.F32, n, batch)
    ts = [to_dev(v) for v in (a, b, c, d)]
    bp.tridiag_batched(*ts, ts[3], n, batch, plan=p)
    torch.cuda.synchronize()
    assert tri_rel_err(ts[3].cpu().numpy(), ref).max() <= 1e-4


def test_decoupled_and_diagonal_systems(bp):
    # a = c = 0 between some rows splits a system into independent blocks;
    # a fully diagonal system is x = d / b
    n, batch = 1024, 4
    a, b, c, d, _ = si.tridiag_f32(batch, n, stream=213)
    a[0, 1::7] = 0.0
    c[0, 0:-1:7] = 0.0
    a[1, :] = 0.0
    c[1, :] = 0.0
    ref = oracle.thomas(a, b, c, d)
    for p in bp.enumerate_plans(bp.OP_TRIDIAG_WM, bp.F32, n):
        x = run_wm(bp, (a, b, c, d), p)
        assert tri_rel_err(x, ref).max() <= 1e-4, p
        np.testing.assert_allclose(x[1], (d[1].astype(np.float64) / b[1]), rtol=1e-6)


@pytest.mark.parametrize("n", [64, 256, 1024, 2048])
def test_full_size_sampled(bp, n):
    batch = (1 << 24) // n
    sysm = si.tridiag_f32(batch, n, stream=230 + n)
    p = bp.query_plan(bp.OP_TRIDIAG_WM, bp.F32, n, batch)
    x = run_wm(bp, sysm, p)
    rows = sample_rows(batch)
    ref = oracle.thomas(*[v[rows] for v in sysm[:4]])
    assert tri_rel_err(x[rows], ref).max() <= 1e-4


def test_invalid_plans_rejected(bp):
    n, batch = 256, 4
    sysm = si.tridiag_f32(batch, n, stream=214)
    good = bp.make_plan(bp.OP_TRIDIAG_WM, n, 4, 1, radix=4, shuffle=1)
    assert bp.check_plan(good, bp.F32, n) == 0
    bad = [
        bp.make_plan(bp.OP_TRIDIAG_WM, n, 4, 1, radix=16, shuffle=1),     # radix not in {2, 4, 8}
        bp.make_plan(bp.OP_TRIDIAG_WM, n, 4, 1, radix=4, shuffle=1, cr_switch=32),  # CR knob on WM
        bp.make_plan(bp.OP_TRIDIAG_WM, n, 1, 1, radix=2, shuffle=1),      # P = 1
        bp.make_plan(bp.OP_TRIDIAG_WM, 16, 4, 8, radix=8, shuffle=1),     # radix > n / P
    ]
    for p in bad:
        with pytest.raises(bp.BplgError):
            run_wm(bp, sysm if p.n == n else si.tridiag_f32(batch, p.n, stream=215), p)


def test_tuners_on_the_wm_space(bp):
    n, batch = 1024, 1 << 12
    sysm = si.tridiag_f32(batch, n, stream=216)
    rows = sample_rows(batch)
    ref = oracle.thomas(*[v[rows] for v in sysm[:4]])
    for method in (bp.TUNE_ANALYTIC, bp.TUNE_LEARNED):
        p, rep = bp.tune_plan(bp.OP_TRIDIAG_WM, bp.F32, n, batch, method, budget=16, seed=3)
        assert p.op == bp.OP_TRIDIAG_WM and p.radix in (2, 4, 8)
        x = run_wm(bp, sysm, p)
        assert tri_rel_err(x[rows], ref).max() <= 1e-4
