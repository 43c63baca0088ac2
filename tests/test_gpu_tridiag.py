"""Tridiagonal CR/PCR parity on the GPU against the float64 Thomas oracle on
the stored float32 systems: relative error <= 1e-4 per system for the float32
solver over every valid plan (threads per system, systems per block,
cr_switch, shuffle PCR, padding) with a ragged batch; <= 1e-12 after the
float64-residual refinement."""
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


def run_tri(bp, sysm, plan=None):
    a, b, c, d = sysm[:4]
    batch, n = b.shape
    ts = [to_dev(v) for v in (a, b, c, d)]
    x = torch.empty_like(ts[0])
    bp.tridiag_batched(*ts, x, n, batch, plan=plan)
    torch.cuda.synchronize()
    return x.cpu().numpy()


def run_refined(bp, sysm, plan=None, max_iter=10, tol=1e-14):
    a, b, c, d = sysm[:4]
    batch, n = b.shape
    ts = [to_dev(v) for v in (a, b, c, d)]
    x = torch.empty((batch, n), dtype=torch.float64, device="cuda")
    it = torch.zeros(batch, dtype=torch.int32, device="cuda")
    bp.tridiag_refined(*ts, x, n, batch, max_iter=max_iter, tol=tol, iters=it, plan=plan)
    torch.cuda.synchronize()
    return x.cpu().numpy(), it.cpu().numpy()


@pytest.mark.parametrize("n", [2, 4, 32, 64, 256, 1024, 2048, 8192])
def test_every_plan_ragged(bp, n):
    batch = 11 if n <= 2048 else 3
    sysm = si.tridiag_f32(batch, n, stream=n)
    ref = oracle.thomas(*sysm[:4])
    plans = bp.enumerate_plans(bp.OP_TRIDIAG, bp.F32, n)
    assert plans
    for p in plans:
        assert tri_rel_err(run_tri(bp, sysm, p), ref).max() <= 1e-4, p


def test_outside_coefficients_never_read(bp):
    n, batch = 256, 5
    a, b, c, d, _ = si.tridiag_f32(batch, n, stream=3)
    a[:, 0] = np.nan
    c[:, -1] = np.nan
    ref = oracle.thomas(a, b, c, d)
    x = run_tri(bp, (a, b, c, d))
    assert np.all(np.isfinite(x)) and tri_rel_err(x, ref).max() <= 1e-4


def test_x_may_alias_d(bp):
    n, batch = 512, 7
    a, b, c, d, _ = si.tridiag_f32(batch, n, stream=4)
    ref = oracle.thomas(a, b, c, d)
    ts = [to_dev(v) for v in (a, b, c, d)]
    bp.tridiag_batched(*ts, ts[3], n, batch)
    torch.cuda.synchronize()
    assert tri_rel_err(ts[3].cpu().numpy(), ref).max() <= 1e-4


@pytest.mark.parametrize("n", [64, 256, 1024, 2048])
def test_full_size_default_plan_sampled(bp, n):
    batch = (1 << 24) // n
    sysm = si.tridiag_f32(batch, n, stream=30 + n)
    x = run_tri(bp, sysm)
    rows = sample_rows(batch)
    ref = oracle.thomas(*[v[rows] for v in sysm[:4]])
    assert tri_rel_err(x[rows], ref).max() <= 1e-4


@pytest.mark.parametrize("n", [32, 64, 256, 1024, 4096])
def test_refined_every_plan(bp, n):
    batch = 5
    sysm = si.tridiag_f32(batch, n, stream=50 + n)
    ref = oracle.thomas(*sysm[:4])
    for p in bp.enumerate_plans(bp.OP_TRIDIAG_REFINED, bp.F32, n):
        x, it = run_refined(bp, sysm, p)
        assert tri_rel_err(x, ref).max() <= 1e-12, p
        assert np.all(it >= 1) and np.all(it <= 10)  # at least one correction: x0 is only float32-accurate


def test_refined_full_config_sampled(bp):
    # n = 1024, 2^14 systems (the precision configuration), default plan
    n, batch = 1024, 1 << 14
    sysm = si.tridiag_f32(batch, n, seed=si.CONFIG_SEEDS["precision"])
    x, it = run_refined(bp, sysm)
    rows = sample_rows(batch)
    ref = oracle.thomas(*[v[rows] for v in sysm[:4]])
    assert tri_rel_err(x[rows], ref).max() <= 1e-12
    # the float32 solve alone is ~1e-7; refinement must have been applied
    assert it.min() >= 1


@pytest.mark.parametrize("P", [8, 16])
def test_refined_wang_mou_full_config_sampled(bp, P):
    # the benchmark's tuned layout (Wang-Mou solves; P = 8 runs the
    # register-capped form) at the full precision configuration
    n, batch = 1024, 1 << 14
    sysm = si.tridiag_f32(batch, n, seed=si.CONFIG_SEEDS["precision"])
    p = bp.make_plan(bp.OP_TRIDIAG_REFINED, n, P, 1, shuffle=1, smem_layout=7, smem_pad=0, cr_switch=32)
    x, it = run_refined(bp, sysm, plan=p, tol=1e-12)
    rows = sample_rows(batch)
    ref = oracle.thomas(*[v[rows] for v in sysm[:4]])
    assert tri_rel_err(x[rows], ref).max() <= 1e-12
    assert it.min() >= 1 and it.max() <= 10


def test_refined_at_the_target_tolerance(bp):
    # stopping at tol = 1e-12 (the benchmark's setting) still meets 1e-12
    n, batch = 1024, 256
    sysm = si.tridiag_f32(batch, n, seed=si.CONFIG_SEEDS["precision"], stream=5)
    ref = oracle.thomas(*sysm[:4])
    x, it = run_refined(bp, sysm, tol=1e-12)
    assert tri_rel_err(x, ref).max() <= 1e-12
    assert it.min() >= 1


def test_refined_with_subnormal_coefficients(bp):
    # systems with subnormal and zero off-diagonal coefficients take the
    # general float -> double widening; every register plan still meets 1e-12
    n, batch = 1024, 6
    a, b, c, d, _ = si.tridiag_f32(batch, n, stream=79)
    a[1, 5::7] = np.float32(3e-39)   # subnormal
    c[3, 2::11] = np.float32(-1e-40)  # subnormal
    a[4, 1::3] = 0.0
    sysm = (a, b, c, d)
    ref = oracle.thomas(a, b, c, d)
    for p in bp.enumerate_plans(bp.OP_TRIDIAG_REFINED, bp.F32, n):
        if p.smem_layout >= 4:
            x, it = run_refined(bp, sysm, p)
            assert tri_rel_err(x, ref).max() <= 1e-12, p


def test_refined_zero_iterations_is_the_float32_solve(bp):
    n, batch = 256, 4
    sysm = si.tridiag_f32(batch, n, stream=77)
    ref = oracle.thomas(*sysm[:4])
    x, it = run_refined(bp, sysm, max_iter=0)
    assert np.all(it == 0)
    assert tri_rel_err(x, ref).max() <= 1e-4


def test_argument_errors(bp):
    v = torch.zeros(8192, dtype=torch.float32, device="cuda")
    # n outside [2, 8192] is refused before any launch (raw pointers)
    for n in (1, 8193):
        assert bp.lib.bplg_tridiag_batched(*([v.data_ptr()] * 5), n, 1, None, None) == bp.ERR_UNSUPPORTED_SIZE
    x64 = torch.zeros(8192, dtype=torch.float64, device="cuda")
    with pytest.raises(bp.BplgError) as e:
        bp.tridiag_refined(v, v, v, v, v, 64, 1)  # x aliases the inputs
    assert e.value.code == bp.ERR_INVALID_ARG
    with pytest.raises(bp.BplgError) as e:
        bp.tridiag_refined(v, v, v, v, x64, 8192, 1)
    assert e.value.code == bp.ERR_UNSUPPORTED_SIZE
    bad = bp.make_plan(bp.OP_TRIDIAG, 64, P=2, spb=1, cr_switch=64, shuffle=1)  # shuffle PCR needs m <= 32
    with pytest.raises(bp.BplgError) as e:
        bp.tridiag_batched(v, v, v, v, v, 64, 1, plan=bad)
    assert e.value.code == bp.ERR_INVALID_PLAN


def test_no_device_error_recorded(bp):
    # every pipelined launch above completed its bounded waits
    assert bp.device_status() == 0


@pytest.mark.parametrize("scale_log2", [100, -100])
def test_systems_scaled_by_powers_of_two(bp, scale_log2):
    """A system multiplied through by 2^100 or 2^-100 (exactly, every
    coefficient and right-hand side) has the same solution: the CR/PCR and
    Wang-Mou solves and the refined solve keep their tolerances at both ends
    of the float32 range the pivots may take."""
    n, batch = 1024, 6
    a, b, c, d, _ = si.tridiag_f32(batch, n, stream=11)
    ref = oracle.thomas(a, b, c, d)
    s = np.float32(2.0 ** scale_log2)
    scaled = tuple(v * s for v in (a, b, c, d))
    assert np.array_equal(oracle.thomas(*scaled), ref)
    assert tri_rel_err(run_tri(bp, scaled), ref).max() <= 1e-4
    wm = bp.query_plan(bp.OP_TRIDIAG_WM, bp.F32, n, batch)
    assert tri_rel_err(run_tri(bp, scaled, wm), ref).max() <= 1e-4
    x, _ = run_refined(bp, scaled, tol=1e-14)
    assert tri_rel_err(x, ref).max() <= 1e-12
