"""Host-side checks of the C ABI (no GPU needed): the library loads and
exports every symbol include/bplg.h declares; occupancy and the analytical
guideline agree with the plain-Python oracle (and so with the paper's
Fig. 2 tables); the Bayesian-optimisation and exhaustive searches behave on
synthetic cost surfaces; argument errors are reported before any device
call."""
import math
import os
import re

import numpy as np
import pytest

import paper_2310_16214_gb300 as bp
from oracle import tuning as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "bplg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bplg_[a-z0-9_]+)\s*\(", src)) - {"bplg_cost_fn"})


def test_every_declared_symbol_is_exported():
    names = header_functions()
    assert len(names) >= 17
    for name in names:
        assert hasattr(bp.lib, name), name
    assert sorted(bp.EXPORTED) == names


def test_version():
    assert bp.version() == 100


def _arch(which):
    return bp.arch_preset(which), (T.TX1 if which == 0 else T.GB300)


@pytest.mark.parametrize("which", [0, 1])
def test_occupancy_parity_with_oracle(which):
    a, oa = _arch(which)
    rng = np.random.default_rng(3 + which)
    for _ in range(2000):
        w = int(rng.integers(1, 33))
        r = int(rng.integers(0, 256))
        s = int(rng.integers(0, 64 * 1024 if which == 0 else 232448))
        assert bp.occupancy(a, w, r, s) == T.occupancy(oa, w, r, s), (w, r, s)


def test_occupancy_fig2a_through_the_abi(golden):
    a = bp.arch_preset(0)
    for w, r, s, occ, blocks, pinned in golden("occupancy_gm20b.txt"):
        if pinned != "yes":
            continue
        W, B = bp.occupancy(a, int(w), int(r), int(s))
        assert (round(100 * W / 64), B) == (int(occ), int(blocks))


def _cands(space):
    return [dict(S=c.S, P=c.P, L=c.L, regs=c.regs, smem=c.smem, radix=c.radix, shuffle=c.shuffle) for c in space]


@pytest.mark.parametrize("op", ["ts", "scan", "fft"])
def test_guideline_parity_on_paper_spaces(op):
    fn = {"ts": T.paper_space_ts, "scan": T.paper_space_scan, "fft": T.paper_space_fft}[op]
    a = bp.arch_preset(0)
    for N in [16, 32, 64, 128, 256, 512, 1024, 2048, 4096]:
        space = fn(N)
        if not space:
            continue
        ref = T.guideline(T.TX1, space, radix_tunable=(op == "fft"))
        got = bp.guideline_select(a, _cands(space), radix_tunable=(op == "fft"))
        assert got == (ref if ref is not None else -1), (op, N)


def test_guideline_reproduces_fig2bcd_through_the_abi(golden):
    a = bp.arch_preset(0)
    fns = {"ts": T.paper_space_ts, "scan": T.paper_space_scan, "fft": T.paper_space_fft}
    for op, N, S, P, L in golden("analytic_tuples_tx1.txt"):
        space = fns[op](int(N))
        i = bp.guideline_select(a, _cands(space), radix_tunable=(op == "fft"))
        c = space[i]
        assert (c.S, c.P, c.L) == (int(S), int(P), int(L)), (op, N)


@pytest.mark.parametrize("which", [0, 1])
def test_guideline_parity_random_lists(which):
    a, oa = _arch(which)
    rng = np.random.default_rng(11 + which)
    for trial in range(300):
        k = int(rng.integers(1, 40))
        space = []
        for _ in range(k):
            P = int(2 ** rng.integers(0, 5))
            L = int(2 ** rng.integers(5, 11))
            space.append(T.Candidate(S=int(rng.integers(0, 4096)), P=P, L=L, regs=int(rng.integers(16, 200)),
                                     smem=int(rng.integers(0, 120000)), radix=int(2 ** rng.integers(1, 5)),
                                     shuffle=int(rng.integers(0, 2))))
        rt = bool(trial % 2)
        ref = T.guideline(oa, space, rt)
        assert bp.guideline_select(a, _cands(space), rt) == (ref if ref is not None else -1)


def test_phi_matches_oracle():
    for e in ([1.0], [1.0, 0.5], [0.9, 0.95, 1.0, 0.7], []):
        assert abs(bp.phi(e) - T.phi(e)) < 1e-15


# ------------------------------------------------ searches on synthetic costs

def synthetic_plans():
    """A plan grid over (P, spb, pad, pattern) -- values only, no device."""
    plans = []
    for P in (1, 2, 4, 8, 16, 32):
        for spb in (1, 2, 4, 8, 16, 32):
            for pad in (0, 1):
                for pat in (0, 1):
                    plans.append(bp.make_plan(bp.OP_SCAN, 1024, P=P, spb=spb, smem_pad=pad, pattern=pat))
    return plans


def quad_cost(p, noise_seed=None):
    # separable quadratic in log2 knobs, optimum at P=8, spb=4, pad=1, pattern=0
    v = 1.0 + 0.3 * (math.log2(p.P) - 3) ** 2 + 0.2 * (math.log2(p.spb) - 2) ** 2 + 0.4 * (1 - p.smem_pad) \
        + 0.1 * p.pattern
    if noise_seed is not None:
        h = hash((p.P, p.spb, p.smem_pad, p.pattern, noise_seed)) % 1000
        v *= 1.0 + 0.01 * (h / 1000.0 - 0.5)
    return v


def test_exhaustive_finds_argmin_and_counts():
    plans = synthetic_plans()
    chosen, rep = bp.tune_plans_cost(plans, quad_cost, bp.TUNE_EXHAUSTIVE)
    assert rep.evaluations == len(plans) == rep.space_size
    best = min(range(len(plans)), key=lambda i: quad_cost(plans[i]))
    assert chosen == best


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_learned_search_near_optimum_within_budget(seed):
    plans = synthetic_plans()
    costs = [quad_cost(p, seed) for p in plans]
    chosen, rep = bp.tune_plans_cost(plans, lambda p: quad_cost(p, seed), bp.TUNE_LEARNED, budget=40, seed=seed)
    assert rep.evaluations <= 40 < len(plans)
    assert costs[chosen] <= 1.05 * min(costs)


def test_learned_search_is_deterministic():
    plans = synthetic_plans()
    seen = []
    for _ in range(2):
        order = []

        def cost(p):
            order.append((p.P, p.spb, p.smem_pad, p.pattern))
            return quad_cost(p, 9)

        chosen, rep = bp.tune_plans_cost(plans, cost, bp.TUNE_LEARNED, budget=30, seed=42)
        seen.append((chosen, tuple(order)))
    assert seen[0] == seen[1]


def test_learned_search_stops_after_the_window_without_progress():
    plans = synthetic_plans()
    chosen, rep = bp.tune_plans_cost(plans, lambda p: 1.0, bp.TUNE_LEARNED, budget=100, seed=1)
    # a flat surface: the initial design (5 points, growing with the square
    # root of the space, at most 24), then the stopping window (8 by default)
    # of evaluations without progress
    n0 = max(5, min(math.ceil(0.6 * math.sqrt(len(plans))), 24))
    assert rep.evaluations == n0 + 8


def test_learned_search_window_of_the_paper():
    # BPLG_BO_WINDOW=5 restores the 5-evaluation window of Section IV-B
    import subprocess
    import sys
    code = ("import math, sys; sys.path.insert(0, %r); import paper_2310_16214_gb300 as bp; "
            "from tests.test_capi_host import synthetic_plans; plans = synthetic_plans(); "
            "c, r = bp.tune_plans_cost(plans, lambda p: 1.0, bp.TUNE_LEARNED, budget=100, seed=1); "
            "n0 = max(5, min(math.ceil(0.6 * math.sqrt(len(plans))), 24)); print(r.evaluations - n0)" % ROOT)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT,
                         env={**os.environ, "BPLG_BO_WINDOW": "5"})
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == "5"


def test_invalid_candidates_are_penalised():
    plans = synthetic_plans()

    def cost(p):
        return -1.0 if p.P == 8 else quad_cost(p)

    chosen, rep = bp.tune_plans_cost(plans, cost, bp.TUNE_EXHAUSTIVE)
    assert plans[chosen].P != 8 and rep.invalid == sum(p.P == 8 for p in plans)
    with pytest.raises(bp.BplgError) as e:
        bp.tune_plans_cost(plans, lambda p: float("inf"), bp.TUNE_EXHAUSTIVE)
    assert e.value.code == bp.ERR_INVALID_PLAN


def test_analytic_method_on_explicit_list():
    space = T.paper_space_fft(1024)
    plans = [bp.make_plan(bp.OP_FFT, 1024, P=c.P, spb=max(1, c.S // 1024)) for c in space]
    chosen, rep = bp.tune_plans_cost(plans, None, bp.TUNE_ANALYTIC, regs=[c.regs for c in space],
                                     smem=[c.smem for c in space], arch=bp.arch_preset(0))
    assert rep.evaluations == 0
    assert chosen == T.guideline(T.TX1, space, True)


# ---------------------------------------------------------- argument errors

def test_argument_errors_before_any_device_call():
    P = bp.lib
    assert P.bplg_scan_batched(0, None, None, 64, 1, None, None) == bp.ERR_INVALID_ARG
    assert P.bplg_scan_batched(7, 16, 16, 64, 1, None, None) == bp.ERR_INVALID_ARG
    assert P.bplg_scan_batched(0, 16, 16, 32769, 1, None, None) == bp.ERR_UNSUPPORTED_SIZE  # above 2^15
    assert P.bplg_scan_batched(0, 16, 16, 64, 0, None, None) == bp.ERR_INVALID_ARG
    assert P.bplg_scan_batched(0, 17, 16, 64, 1, None, None) == bp.ERR_INVALID_ARG  # misaligned
    assert P.bplg_fft_batched(16, 16, 64, 1, 0, None, None) == bp.ERR_INVALID_ARG
    assert P.bplg_fft_batched(16, 16, 1 << 25, 1, -1, None, None) == bp.ERR_UNSUPPORTED_SIZE
    assert P.bplg_fft_batched(16, 16, (1 << 23) + 1, 1, -1, None, None) == bp.ERR_UNSUPPORTED_SIZE  # Bluestein limit
    assert P.bplg_tridiag_batched(16, 16, 16, 16, 16, 1, 1, None, None) == bp.ERR_UNSUPPORTED_SIZE
    assert P.bplg_tridiag_batched(16, 16, 16, None, 16, 64, 1, None, None) == bp.ERR_INVALID_ARG
    assert P.bplg_tridiag_batched(16, 16, 16, 16, 16, 1 << 14, 1, None, None) == bp.ERR_UNSUPPORTED_SIZE
    assert P.bplg_tridiag_refined(16, 16, 16, 16, 4096, 64, 1, 65, 1e-14, None, None, None) == bp.ERR_INVALID_ARG
    assert P.bplg_tridiag_refined(16, 16, 16, 16, 4096, 64, 1, 5, -1.0, None, None, None) == bp.ERR_INVALID_ARG
    assert P.bplg_tridiag_refined(16, 16, 16, 16, 16, 64, 1, 5, 1e-14, None, None, None) == bp.ERR_INVALID_ARG
    assert bp.last_error()


def test_no_device_is_reported_not_faked():
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    rc = bp.lib.bplg_scan_batched(0, 4096, 4096, 64, 1, None, None)
    assert rc == bp.ERR_NO_DEVICE


def test_grid_above_the_launch_limit_is_rejected_before_any_device_call():
    """A batch that would need more than 2^31 - 1 blocks under the caller's
    plan is refused on the host (nothing is enqueued); one block fewer gets
    past that check (and then, on a machine without a GPU, stops at the
    device query)."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present: the just-below-the-limit calls would reach it")
    except ImportError:
        pass
    import ctypes
    P = bp.lib
    scan = bp.make_plan(bp.OP_SCAN, 32, P=1, spb=1)  # one 32-element problem per block
    assert P.bplg_scan_batched(0, 16, 16, 32, 1 << 31, ctypes.byref(scan), None) == bp.ERR_UNSUPPORTED_SIZE
    assert "2^31" in bp.last_error()
    assert P.bplg_scan_batched(0, 16, 16, 32, (1 << 31) - 1, ctypes.byref(scan), None) == bp.ERR_NO_DEVICE
    fft = bp.make_plan(bp.OP_FFT, 64, P=2, spb=1)
    assert P.bplg_fft_batched(16, 16, 64, 1 << 31, -1, ctypes.byref(fft), None) == bp.ERR_UNSUPPORTED_SIZE
    assert P.bplg_fft_batched_noalloc(16, 16, 64, 1 << 31, -1, ctypes.byref(fft), None) == bp.ERR_UNSUPPORTED_SIZE
    tri = bp.make_plan(bp.OP_TRIDIAG, 64, P=2, spb=1, cr_switch=32, shuffle=1)
    assert P.bplg_tridiag_batched(16, 16, 16, 16, 16, 64, 1 << 33, ctypes.byref(tri), None) == bp.ERR_UNSUPPORTED_SIZE


# ------------------------------------------------- GB300 cost model (MODEL)

def _scan_space(n):
    """Every (P, spb) scan plan of size n with a plausible register count
    (grows with the elements each thread holds) and no shared memory."""
    plans, regs = [], []
    for P in (1, 2, 4, 8, 16, 32):
        tps = n // P
        if tps < 1 or tps > 1024:
            continue
        for L in (32, 64, 128, 256, 512, 1024):
            if L < tps or L % tps:
                continue
            plans.append(bp.make_plan(bp.OP_SCAN, n, P=P, spb=L // tps))
            regs.append(16 + P + (16 if P == 32 else 0))
    return plans, regs


def test_cost_model_evaluates_nothing_and_is_deterministic():
    plans, regs = _scan_space(1024)
    calls = []
    a = bp.arch_preset(1)
    c1, rep = bp.tune_plans_cost(plans, lambda p: calls.append(1) or 1.0, bp.TUNE_MODEL, regs=regs,
                                 smem=[0] * len(plans), arch=a)
    c2, _ = bp.tune_plans_cost(plans, None, bp.TUNE_MODEL, regs=regs, smem=[0] * len(plans), arch=a)
    assert calls == [] and rep.evaluations == 0 and c1 == c2 and 0 <= c1 < len(plans)


def test_cost_model_premises_on_a_scan_space():
    """Coalescing and bytes in flight: one element per thread cannot keep
    HBM busy, and a block of one warp per 32 elements pays the launch rate;
    the model picks several elements per thread and blocks of more than one
    warp."""
    plans, regs = _scan_space(1024)
    c, _ = bp.tune_plans_cost(plans, None, bp.TUNE_MODEL, regs=regs, smem=[0] * len(plans), arch=bp.arch_preset(1))
    assert plans[c].P >= 4 and plans[c].L >= 64


def test_cost_model_skips_plans_that_cannot_launch():
    plans, regs = _scan_space(256)
    regs = [300 if p.P >= 4 else r for p, r in zip(plans, regs)]  # above the 255-register limit
    c, _ = bp.tune_plans_cost(plans, None, bp.TUNE_MODEL, regs=regs, smem=[0] * len(plans), arch=bp.arch_preset(1))
    assert plans[c].P < 4


def test_cost_model_prefers_padded_exchanges():
    """Bank conflicts: of two FFT plans that differ only in the padding of
    the shared-memory exchange, the padded one is modelled faster."""
    base = dict(P=16, spb=1, radix=16, smem_layout=0, io=0)
    plans = [bp.make_plan(bp.OP_FFT, 4096, smem_pad=0, **base), bp.make_plan(bp.OP_FFT, 4096, smem_pad=1, **base)]
    c, _ = bp.tune_plans_cost(plans, None, bp.TUNE_MODEL, regs=[60, 60], smem=[32768, 34816], arch=bp.arch_preset(1))
    assert c == 1
