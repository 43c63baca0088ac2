"""Tuners against exhaustive search on the GPU (Section VI's comparison):
the learned-cost-model search lands within 5 % of the exhaustive best on a
small space, and the GB300 cost model (no evaluation) within 15 % on spaces
of every operation, the two-kernel FFT's joint (split, columns, rows per
block) space included.  Times are re-measured back to back (median of 30
launches) so the comparison does not rest on the searches' own samples."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_16214_gb300 as bp
    return bp


def _e(bp, plan, best_plan, dt, n, batch):
    t = bp.time_plan(plan, dt, n, batch, 30)
    tb = bp.time_plan(best_plan, dt, n, batch, 30)
    return min(t, tb) / t


def test_learned_within_five_percent_of_exhaustive_scan_1024(bp):
    n, batch = 1024, 1 << 16
    pe, re_ = bp.tune_plan(bp.OP_SCAN, bp.I32, n, batch, bp.TUNE_EXHAUSTIVE)
    assert re_.evaluations == re_.space_size > 0
    pl, rl = bp.tune_plan(bp.OP_SCAN, bp.I32, n, batch, bp.TUNE_LEARNED, budget=40, seed=1)
    assert 0 < rl.evaluations <= min(40, rl.space_size)
    assert _e(bp, pl, pe, bp.I32, n, batch) >= 0.95


@pytest.mark.parametrize("case", [("scan", 8192, 1 << 13), ("fft", 1024, 1 << 14), ("tridiag", 256, 1 << 16),
                                  ("tridiag_wm", 1024, 1 << 14), ("refined", 1024, 1 << 13),
                                  ("fft", 1 << 18, 1 << 6)])
def test_cost_model_near_exhaustive(bp, case):
    name, n, batch = case
    op, dt = {"scan": (bp.OP_SCAN, bp.I32), "fft": (bp.OP_FFT, bp.F32), "tridiag": (bp.OP_TRIDIAG, bp.F32),
              "tridiag_wm": (bp.OP_TRIDIAG_WM, bp.F32), "refined": (bp.OP_TRIDIAG_REFINED, bp.F32)}[name]
    pm, rm = bp.tune_plan(op, dt, n, batch, bp.TUNE_MODEL)
    assert rm.evaluations == 0
    pe, _ = bp.tune_plan(op, dt, n, batch, bp.TUNE_EXHAUSTIVE)
    assert _e(bp, pm, pe, dt, n, batch) >= 0.85, (pm, pe)


def test_default_plan_is_the_cost_model_plan(bp):
    """A plan-less call's plan (bplg_query_plan with nothing cached) is the
    cost model's choice for that size."""
    n = 4096  # modelled, like every default plan, for a batch of 2^24 / n problems
    q = bp.query_plan(bp.OP_TRIDIAG_WM, bp.F32, n, 1 << 12)
    pm, _ = bp.tune_plan(bp.OP_TRIDIAG_WM, bp.F32, n, 1 << 12, bp.TUNE_MODEL)
    assert q.key() == pm.key()
