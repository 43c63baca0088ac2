#!/usr/bin/env python3
"""Benchmark of the batched parallel-prefix hot path on one GB300 per rank.

One step = one pass of every data-path row over synthetic batches shaped like
the paper's workloads (Section VI: batches of problems of power-of-two size,
float32, data resident on the GPU):

  fft      complex64 Stockham FFT, forward and inverse, N in {16, 64, 256,
           1024, 4096}, batch = 2^24 / N signals each
  tridiag  float32 CR/PCR solve, n in {64, 256, 1024, 2048}, 2^24 unknowns each
  refined  float64-residual refined solve, n = 1024, 2^14 systems, stopping
           once a correction is below 1e-12 max|x|
  scan     inclusive sum scan, int32 and float32, n in {64, 1024, 8192},
           2^26 elements each
  uneven   4096 int32 scans + 4096 forward FFTs + 4096 tridiagonal systems,
           sizes 2^e with e uniform on {5..13}, as one graph launch

Every buffer pair is larger than the 129 MB L2, and consecutive launches touch
different buffers, so no L2 flush is needed between them.  `value` is the
total elements processed per second (Gelem/s) over all ranks.  Plans: every
row is tuned before the timed region by the library's learned-cost-model
(Bayesian optimisation) tuner (--plans learned, the default), or taken from
bplg_query_plan (--plans query: cached tuned plan, else the analytical
guideline).

--impl reference times the CPU oracle (test infrastructure) on a bounded
sample of the same workload and prints the same line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import seeded_inputs as si  # noqa: E402

FFT_SIZES = [16, 64, 256, 1024, 4096]
TRI_SIZES = [64, 256, 1024, 2048]
SCAN_SIZES = [64, 1024, 8192]
FFT_TOTAL = 1 << 24
TRI_TOTAL = 1 << 24
SCAN_TOTAL = 1 << 26
REF_N, REF_BATCH = 1024, 1 << 14
UNEVEN_COUNT = 4096
REF_TOL = 1e-12  # refinement stops once a correction is below 1e-12 max|x|, the stated accuracy target

METRIC = "batched scan/FFT/tridiag Gelem/s, %HBM roofline; tuned vs exhaustive-best"
WORKLOAD = ("fft c2c fwd+inv N=16..4096 batch=2^24/N; tridiag CR/PCR n=64..2048 2^24 unknowns; "
            "refined n=1024 x 2^14; scan i32+f32 n=64,1024,8192 x 2^26; "
            "uneven 3x4096 problems n=2^U{5..13} in one graph launch")


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
# the kernel as it stands, from one ncu capture of the same row at half the
# batch, doubled; keyed by row and plan.  A launch whose plan was not captured
# reports null.
NCU_TRAFFIC = {
    # DRAM read + write of one half-size launch of the kernel as it stands,
    # doubled (the rest of x is still in L2 at kernel end).  Layout 6, P = 16:
    # tridiag_refined_reg_kernel
    ("refined_1024", (("P", 16), ("L", 64), ("spb", 1), ("shuffle", 1), ("pattern", 0), ("smem_layout", 6),
                      ("smem_pad", 0), ("io", 0), ("cr_switch", 32))): 2 * (134331648 + 26756608),
    # the Wang-Mou layout (7), P = 8: tridiag_refined_reg_kernel_mb<..., 7> (72
    # registers, seven threads-per-system bits at compile time)
    ("refined_1024", (("P", 8), ("L", 128), ("spb", 1), ("shuffle", 1), ("pattern", 0), ("smem_layout", 7),
                      ("smem_pad", 0), ("io", 0), ("cr_switch", 32))): 2 * (134336768 + 28204288),
}

# FP64 issue rate of one SM: 2 double-precision fused multiply-adds per clock
# (the GB300 FP64 pipe; 152 SMs x 2 x 2 flop x 2.07 GHz = 1.26 TFLOP/s).
FP64_FMA_PER_SM_CLK = 2
DEFAULT_SM_MHZ = 2070.0


def plan_key(plan):
    if plan is None:
        return None
    d = plan.as_dict()
    return tuple((k, d[k]) for k in ("P", "L", "spb", "shuffle", "pattern", "smem_layout", "smem_pad", "io",
                                     "cr_switch"))


def measure_fp64_peak(torch):
    """The FP64 pipe's throughput measured on this GPU: eight independent
    chains of double-precision fused multiply-adds per thread on every SM at
    full residency (extref_fp64_fma, a measurement kernel outside the
    library), best of 5 event-timed launches of about 16 ms each.  Returns
    (TFLOP/s, description) or (None, reason)."""
    import ctypes
    try:
        lib = ctypes.CDLL(os.path.join(ROOT, "paper_2310_16214_gb300", "_lib", "libbplg_extref.so"))
        lib.extref_fp64_fma.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
        tf, ms = ctypes.c_double(), ctypes.c_double()
        iters = 4096
        rc = lib.extref_fp64_fma(iters, 5, ctypes.byref(tf), ctypes.byref(ms),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        if rc != 0:
            return None, "extref_fp64_fma returned %d" % rc
        return tf.value, ("measured: DFMA chains (8 per thread, %d iterations, SMs x 8 blocks of 256 threads), "
                          "best of 5 launches of %.1f ms" % (iters, ms.value))
    except Exception as exc:
        return None, "unavailable: %s" % str(exc)[:120]


def dominant_roofline(dom, dom_ms, peak, peak_kind, refined_iters, clocks, fp64_peak=None):
    """Roofline of the step's longest launch.

    The refined solve is bound by the FP64 pipe, not by HBM: its algorithmic
    work is 3 FP64 fused multiply-adds (6 flop) per unknown for every residual
    and one FP64 add per unknown for every correction, with one residual more
    than corrections (the last residual proves convergence).  Its peak is the
    FP64 rate measured by measure_fp64_peak (else derived from the SM count,
    2 FP64 FMA per SM per clock and the maximum SM clock).  Every other row
    moves its algorithmic bytes once and is reported against HBM bandwidth."""
    traffic = NCU_TRAFFIC.get((dom["name"], plan_key(dom["plan"])))
    gbs = dom["bytes"] / (dom_ms * 1e-3) / 1e9
    if dom["op"] == "refined" and refined_iters is not None:
        import torch
        c = refined_iters["mean"]
        flops = dom["elems"] * (6.0 * (c + 1.0) + c)
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        mhz = clocks.get("sm_max_mhz") or DEFAULT_SM_MHZ
        derived = sms * FP64_FMA_PER_SM_CLK * 2 * mhz * 1e6 / 1e12
        if fp64_peak and fp64_peak[0]:
            fp64, kind = fp64_peak[0], fp64_peak[1]
        else:
            fp64 = derived
            kind = "derived (%d SMs x %d FP64 FMA/clk x 2 flop x %.0f MHz); %s" % (
                sms, FP64_FMA_PER_SM_CLK, mhz, fp64_peak[1] if fp64_peak else "not measured")
        achieved = flops / (dom_ms * 1e-3) / 1e12
        return {"bound": "alu", "pipe": "fp64", "kernel": dom["name"], "achieved": round(achieved, 4),
                "peak": round(fp64, 4), "peak_kind": kind, "derived_peak": round(derived, 4),
                "unit": "TFLOP/s", "frac": round(achieved / fp64, 4), "traffic": traffic,
                "traffic_note": ("DRAM read + write of one ncu capture of this kernel and plan on the half-size "
                                 "case, doubled; part of x was still in L2 when that kernel ended, so the write "
                                 "side is below the algorithmic 8 B per unknown") if traffic else None,
                "algorithmic_flops": flops, "algorithmic_bytes": dom["bytes"], "launch_ms": round(dom_ms, 5),
                "hbm": {"achieved": round(gbs, 1), "peak": peak, "peak_kind": peak_kind, "frac": round(gbs / peak, 4)}}
    return {"bound": "hbm", "kernel": dom["name"], "achieved": round(gbs, 1), "peak": peak,
            "peak_kind": peak_kind, "unit": "GB/s", "frac": round(gbs / peak, 4),
            "traffic": traffic, "algorithmic_bytes": dom["bytes"], "launch_ms": round(dom_ms, 5)}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 10 ms from before
    the warm-up steps until after the timed region.  Every reading carries the
    host time it arrived; the summary keeps the readings that arrived while
    the timed region ran, and when the region is shorter than the sampling
    period (a few dozen milliseconds) the last reading before it and the
    first after it, taken while the warm-up steps and the timed steps kept
    the GPU busy ("window": "bracketing")."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 10

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []  # (host time, csv line)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", str(self.PERIOD_MS)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
            return
        # the sampler's start-up (NVML initialisation) can hold the GPU for
        # tens of milliseconds: wait for its first reading before timing
        t0 = time.time()
        while not self.lines and time.time() - t0 < 10.0:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    @staticmethod
    def _parse(line):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            return None
        try:
            sm, smax = float(parts[1]), float(parts[2])
        except ValueError:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = {name for name, v in zip(names, parts[5:9]) if v.lower().startswith("active")}
        return sm, smax, reasons

    def stop(self, t_begin=None, t_end=None):
        """Summary of the readings between host times t_begin and t_end."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(2.5 * self.PERIOD_MS / 1e3)  # the first reading after the region
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [(t, r) for t, r in ((t, self._parse(line)) for t, line in list(self.lines)) if r is not None]
        window = "timed region"
        if t_begin is None:
            chosen = rows
        else:
            chosen = [(t, r) for t, r in rows if t_begin <= t <= t_end]
            if not chosen:
                before = [(t, r) for t, r in rows if t < t_begin]
                after = [(t, r) for t, r in rows if t > t_end]
                chosen = before[-1:] + after[:1]
                window = "bracketing"
        sm = [r[0] for _, r in chosen]
        smax = max((r[1] for _, r in chosen), default=None)
        reasons = set()
        for _, r in chosen:
            reasons |= r[2]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm), "window": window,
                "period_ms": self.PERIOD_MS, "readings_total": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest value of x over all ranks (the slowest rank's time); the
    only collective of the bench, outside the timed region."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, elems_per_rank: int, step_ms: float) -> float:
    """Whole-job throughput in Gelem/s: every rank runs its own replica of the
    per-GPU workload (weak scaling), all in the same max-over-ranks step time."""
    return world * elems_per_rank / (step_ms * 1e-3) / 1e9


# ----------------------------------------------------------------- workload

class Workload:
    """Device buffers for every row of the step, filled from the seeded generators,
    and the plan each row runs with."""

    def __init__(self, torch, bp, dev, scale: float = 1.0, rows=None, plans="learned", plan_json=None,
                 seed: int = 1):
        self.torch, self.bp, self.dev = torch, bp, dev
        self.items = []
        self.rows = set(rows) if rows else None
        self.plans_mode = plans
        self.fixed = plan_json or {}
        self.seed = seed
        self.tuning = {"mode": plans, "seconds": 0.0, "evaluations": 0}
        self.learned = {}  # row -> (plan, BO evaluations, space size)
        t = torch
        for n in FFT_SIZES:
            batch = max(1, int(FFT_TOTAL * scale) // n)
            if not self._want("fft_fwd_%d" % n) and not self._want("fft_inv_%d" % n):
                continue
            z = si.fft_c64(batch, n, stream=100 + n)
            zin = t.from_numpy(z.view(np.float32).reshape(-1)).to(dev)
            zout = t.empty_like(zin)
            for direction, tag in ((-1, "fwd"), (1, "inv")):
                name = "fft_%s_%d" % (tag, n)
                if not self._want(name):
                    continue
                p = self._plan(name, bp.OP_FFT, bp.F32, n, batch)
                self._add(name, "fft", n, batch, batch * n, 16 * batch * n,
                          (lambda zi=zin, zo=zout, n=n, b=batch, d=direction, p=p:
                           bp.fft_batched(zi, zo, n, b, d, plan=p)), [zin], [zout], p)
        for n in TRI_SIZES:
            name = "tridiag_%d" % n
            if not self._want(name):
                continue
            batch = max(1, int(TRI_TOTAL * scale) // n)
            a, b, c, d, _ = si.tridiag_f32(batch, n, stream=200 + n)
            ts = [t.from_numpy(v).to(dev) for v in (a, b, c, d)]
            x = t.empty_like(ts[0])
            p = self._plan(name, bp.OP_TRIDIAG, bp.F32, n, batch)
            self._add(name, "tridiag", n, batch, batch * n, 20 * batch * n,
                      (lambda ts=ts, x=x, n=n, b=batch, p=p: bp.tridiag_batched(*ts, x, n, b, plan=p)), ts, [x], p)
        # Wang-Mou rows: only when named in --rows (the step's tridiagonal
        # rows are the CR/PCR hybrid the configuration names)
        for n in TRI_SIZES:
            name = "tridiag_wm_%d" % n
            if self.rows is None or name not in self.rows:
                continue
            batch = max(1, int(TRI_TOTAL * scale) // n)
            a, b, c, d, _ = si.tridiag_f32(batch, n, stream=200 + n)
            ts = [t.from_numpy(v).to(dev) for v in (a, b, c, d)]
            x = t.empty_like(ts[0])
            p = self._plan(name, bp.OP_TRIDIAG_WM, bp.F32, n, batch)
            self._add(name, "tridiag_wm", n, batch, batch * n, 20 * batch * n,
                      (lambda ts=ts, x=x, n=n, b=batch, p=p: bp.tridiag_batched(*ts, x, n, b, plan=p)), ts, [x], p)
        name = "refined_%d" % REF_N
        if self._want(name):
            batch = max(1, int(REF_BATCH * scale))
            a, b, c, d, _ = si.tridiag_f32(batch, REF_N, seed=si.CONFIG_SEEDS["precision"])
            ts = [t.from_numpy(v).to(dev) for v in (a, b, c, d)]
            x64 = t.empty((batch, REF_N), dtype=t.float64, device=dev)
            self.iters = t.zeros(batch, dtype=t.int32, device=dev)
            p = self._plan(name, bp.OP_TRIDIAG_REFINED, bp.F32, REF_N, batch)
            self._add(name, "refined", REF_N, batch, batch * REF_N, 24 * batch * REF_N,
                      (lambda ts=ts, x=x64, b=batch, p=p, it=self.iters:
                       bp.tridiag_refined(*ts, x, REF_N, b, tol=REF_TOL, iters=it, plan=p)), ts, [x64], p)
        name = "uneven"
        if self._want(name) and scale >= 1.0:
            self._add_uneven(torch, bp, dev)
        for dname, dt, gen in (("i32", bp.I32, lambda b, n: si.scan_i32(b, n, stream=300 + n)),
                               ("f32", bp.F32, lambda b, n: si.scan_f32(b, n, stream=400 + n))):
            for n in SCAN_SIZES:
                name = "scan_%s_%d" % (dname, n)
                if not self._want(name):
                    continue
                batch = max(1, int(SCAN_TOTAL * scale) // n)
                xin = t.from_numpy(gen(batch, n)).to(dev)
                xout = t.empty_like(xin)
                p = self._plan(name, bp.OP_SCAN, dt, n, batch)
                self._add(name, "scan_" + dname, n, batch, batch * n, 8 * batch * n,
                          (lambda xi=xin, xo=xout, n=n, b=batch, p=p, dt=dt:
                           bp.scan_batched(xi, xo, n, b, dtype=dt, plan=p)), [xin], [xout], p)

    def _add_uneven(self, torch, bp, dev):
        """4096 int32 scans + 4096 complex64 FFTs + 4096 float32 tridiagonal
        systems, sizes 2^e with e uniform on {5..13}: one graph launch."""
        count = UNEVEN_COUNT
        seed = si.CONFIG_SEEDS["uneven"]
        sizes = si.uneven_sizes(3 * count, seed)
        # one backing buffer per kind, items at 16-byte-aligned offsets
        ns = [int(v) for v in sizes]
        tot = [sum(ns[:count]), sum(ns[count:2 * count]), sum(ns[2 * count:])]
        scan_in = torch.from_numpy(si.scan_i32(1, tot[0], seed=seed, stream=1)[0]).to(dev)
        scan_out = torch.empty_like(scan_in)
        z = si.fft_c64(1, tot[1], seed=seed, stream=2)[0]
        fft_in = torch.from_numpy(z.view(np.float32)).to(dev)
        fft_out = torch.empty_like(fft_in)
        a, b, c, d = (t.reshape(-1) for t in si.tridiag_f32(1, tot[2], seed=seed, stream=3)[:4])
        # each tridiagonal item is its own system (the kernels never read its a[0] and c[n-1])
        tri = [torch.from_numpy(v.copy()).to(dev) for v in (a, b, c, d)]
        tri_x = torch.empty_like(tri[0])
        items, nbytes = [], 0
        off = 0
        for n in ns[:count]:
            items.append({"op": bp.OP_SCAN, "n": n, "dtype": bp.I32, "in": [scan_in[off:off + n]],
                          "out": scan_out[off:off + n]})
            off += n
            nbytes += 8 * n
        off = 0
        for n in ns[count:2 * count]:
            items.append({"op": bp.OP_FFT, "n": n, "dir": -1, "in": [fft_in[2 * off:2 * (off + n)]],
                          "out": fft_out[2 * off:2 * (off + n)]})
            off += n
            nbytes += 16 * n
        off = 0
        for n in ns[2 * count:]:
            items.append({"op": bp.OP_TRIDIAG, "n": n, "in": [t[off:off + n] for t in tri],
                          "out": tri_x[off:off + n]})
            off += n
            nbytes += 20 * n
        ub = bp.UnevenBatch(items)
        self.uneven = ub
        elems = sum(ns)
        self._add("uneven", "uneven", 0, 3 * count, elems, nbytes, (lambda ub=ub: ub.launch()),
                  [scan_in, fft_in] + tri, [scan_out, fft_out, tri_x], bp.Plan())

    def _want(self, name):
        return self.rows is None or name in self.rows

    def _plan(self, name, op, dtype, n, batch):
        bp = self.bp
        if name in self.fixed:
            p = bp.make_plan(op, n, self.fixed[name]["P"], self.fixed[name]["spb"],
                             **{k: v for k, v in self.fixed[name].items() if k not in ("P", "spb", "op", "n", "L", "S")})
            return p
        if self.plans_mode == "query":
            return bp.query_plan(op, dtype, n, batch)
        t0 = time.time()
        p, rep = bp.tune_plan(op, dtype, n, batch, bp.TUNE_LEARNED, budget=40, seed=self.seed)
        self.tuning["seconds"] += time.time() - t0
        self.tuning["evaluations"] += rep.evaluations
        self.learned[name] = (p, rep.evaluations, rep.space_size)
        return p

    def _add(self, name, op, n, batch, elems, nbytes, fn, ins, outs, plan):
        self.items.append(dict(name=name, op=op, n=n, batch=batch, elems=elems, bytes=nbytes, fn=fn,
                               ins=ins, outs=outs, plan=plan))

    @property
    def elems(self):
        return sum(i["elems"] for i in self.items)


def run_ours(args):
    import torch
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    import paper_2310_16214_gb300 as bp

    plan_json = json.loads(args.plan_json) if args.plan_json else None
    wl = Workload(torch, bp, dev, scale=args.scale, rows=args.rows.split(",") if args.rows else None,
                  plans=args.plans, plan_json=plan_json, seed=args.seed)
    stream = torch.cuda.current_stream()

    def make_events(k):
        return {it["name"]: [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                             for _ in range(k)] for it in wl.items}

    def step(evs=None, idx=0):
        for it in wl.items:
            if evs is None:
                it["fn"]()
                continue
            e0, e1 = evs[it["name"]][idx]
            e0.record(stream)
            it["fn"]()
            e1.record(stream)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # every event of the timed region exists before it starts, and the first
    # warm-up step records events too, so no first-use cost lands in a timed
    # launch.  The clock sampler runs from before the warm-up steps to after
    # the timed region.
    fp64_peak = measure_fp64_peak(torch) if "refined_%d" % REF_N in [it["name"] for it in wl.items] else None
    ev = make_events(args.steps)
    ev_warm = make_events(1)
    sampler = ClockSampler(local if world > 1 else 0)
    sampler.start()
    for w in range(args.warmup):
        step(ev_warm if w == 0 else None)
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")  # lets a profiler keep exactly the timed launches
    host_begin = time.time()
    t0.record(stream)
    for k in range(args.steps):
        step(ev, k)
    t1.record(stream)
    torch.cuda.nvtx.range_pop()
    barrier()
    host_end = time.time()
    clocks = sampler.stop(host_begin, host_end)
    total_ms = max_over_ranks(t0.elapsed_time(t1), world, dev)

    per_item, per_item_median, per_item_pct = {}, {}, {}
    for it in wl.items:
        ms = sorted(a.elapsed_time(b) for a, b in ev[it["name"]])
        per_item[it["name"]] = statistics.mean(ms)
        per_item_median[it["name"]] = statistics.median(ms)
        per_item_pct[it["name"]] = (ms[int(0.1 * (len(ms) - 1))], ms[int(0.9 * (len(ms) - 1))])
    per_op = {}
    for it in wl.items:
        d = per_op.setdefault(it["op"], {"ms": 0.0, "elems": 0, "bytes": 0})
        d["ms"] += per_item[it["name"]]
        d["elems"] += it["elems"]
        d["bytes"] += it["bytes"]
    peak, peak_kind = read_peaks()
    for k, d in per_op.items():
        d["gelem_s"] = d["elems"] / (d["ms"] * 1e-3) / 1e9
        d["gb_s"] = d["bytes"] / (d["ms"] * 1e-3) / 1e9
        d["hbm_frac"] = d["gb_s"] / peak
        d["ms"] = round(d["ms"], 4)
    refined_iters = None
    if hasattr(wl, "iters"):
        it_np = wl.iters.cpu().numpy()
        refined_iters = {"mean": round(float(it_np.mean()), 3), "max": int(it_np.max()), "min": int(it_np.min())}
    # dominant kernel: the launch with the largest share of the step
    dom = max(wl.items, key=lambda it: per_item[it["name"]])
    roofline = dominant_roofline(dom, per_item[dom["name"]], peak, peak_kind, refined_iters, clocks, fp64_peak)
    step_ms = total_ms / args.steps
    value = job_value(world, wl.elems, step_ms)
    # kernels launched per step: one per row, three for the uneven batch's
    # graph (one persistent kernel per operation)
    launches_per_step = sum(3 if it["op"] == "uneven" else 1 for it in wl.items)
    items_out = {it["name"]: {"ms": round(per_item[it["name"]], 5),
                              "median_ms": round(per_item_median[it["name"]], 5),
                              "p10_ms": round(per_item_pct[it["name"]][0], 5),
                              "p90_ms": round(per_item_pct[it["name"]][1], 5),
                              "mrows_s": round(it["batch"] / (per_item[it["name"]] * 1e-3) / 1e6, 1),
                              "gflops": (round(5 * it["n"] * math.log2(it["n"]) * it["batch"]
                                               / (per_item[it["name"]] * 1e-3) / 1e9, 1) if it["op"] == "fft" else None),
                              "gb_s": round(it["bytes"] / (per_item[it["name"]] * 1e-3) / 1e9, 1),
                              "plan": {k: v for k, v in it["plan"].as_dict().items()
                                       if k in ("P", "L", "spb", "smem_layout", "smem_pad", "io", "cr_switch",
                                                "shuffle", "pattern")
                                       or (k == "radix" and it["op"] == "tridiag_wm")}}
                 for it in wl.items}

    ext = None
    if rank == 0 and not args.no_ext and wl.items:
        try:
            ext = external_refs(torch, per_item, peak)
        except Exception as exc:  # the references are context; their absence does not fail the bench
            ext = {"unavailable": str(exc)[:200]}
    e2e = measure_e2e(torch, wl, stream, args) if rank == 0 and not args.no_e2e else None
    cpu = cpu_baseline(args) if (rank == 0 and world == 1 and not args.no_cpu) else None
    tuning = None
    if rank == 0 and not args.no_tuning and args.plans == "learned" and wl.learned:
        try:
            tuning = tuning_quality(bp, wl)
        except Exception as exc:  # reported, never fatal to the bench line
            tuning = {"unavailable": str(exc)[:200]}
    precision = None
    if rank == 0 and not args.no_precision:
        try:
            precision = precision_quality(bp, torch, peak)
        except Exception as exc:  # reported, never fatal to the bench line
            precision = {"unavailable": str(exc)[:200]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "Gelem/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (fft, tridiag, scan f32), i32 (scan), f64 residual (refined)",
            "data": "synthetic (seeded SplitMix64, paper-shaped batches)",
            "config": {"workload": WORKLOAD, "elems_per_step_per_gpu": wl.elems,
                       "l2": "inputs larger than L2 (every buffer pair > 129 MB), no flush",
                       "plans": wl.tuning,
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": roofline, "per_op": per_op, "per_launch": items_out,
            "gpu_launches": launches_per_step * args.steps, "clocks": clocks, "refined_corrections": refined_iters,
            "e2e": e2e, "cpu_baseline": cpu, "external": ext, "tuning": tuning, "precision": precision,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def tuning_quality(bp, wl, reps: int = 30):
    """Tuned vs exhaustive-best (Section VI) for every op and size of the
    timed step (forward FFTs, CR/PCR solves, the refined solve, both scans):
    the plan of the GB300 cost model (BPLG_TUNE_MODEL, no evaluation), of the
    paper's guideline (BPLG_TUNE_ANALYTIC, no evaluation), of the learned
    tuner the step runs with (Bayesian optimisation), and of exhaustive search
    over the same space, re-timed back to back by bplg_time_plan (median of
    `reps` launches each, on library-owned buffers of the row's shape).
    e = t_best / t_plan with t_best the fastest of the four; Phi per op is
    the harmonic mean of e over its sizes."""
    kinds = {"fft": (bp.OP_FFT, bp.F32), "tridiag": (bp.OP_TRIDIAG, bp.F32),
             "refined": (bp.OP_TRIDIAG_REFINED, bp.F32), "scan_i32": (bp.OP_SCAN, bp.I32),
             "scan_f32": (bp.OP_SCAN, bp.F32)}
    t0 = time.time()
    rows, exh_evals = [], 0
    for it in wl.items:
        name, op_name = it["name"], it["op"]
        if op_name == "fft" and name.startswith("fft_inv"):
            continue  # the tuners time forward transforms
        if op_name not in kinds or name not in wl.learned:
            continue
        op, dt = kinds[op_name]
        n, batch = it["n"], it["batch"]
        pl, bo_evals, space = wl.learned[name]
        pm, _ = bp.tune_plan(op, dt, n, batch, bp.TUNE_MODEL)
        pg, _ = bp.tune_plan(op, dt, n, batch, bp.TUNE_ANALYTIC)
        pe, rep_e = bp.tune_plan(op, dt, n, batch, bp.TUNE_EXHAUSTIVE)
        exh_evals += rep_e.evaluations
        times = {}
        for key, p in (("model", pm), ("analytic", pg), ("learned", pl), ("exhaustive", pe)):
            same = [k for k, q in (("model", pm), ("analytic", pg), ("learned", pl), ("exhaustive", pe))
                    if k in times and q.key() == p.key()]
            times[key] = times[same[0]] if same else bp.time_plan(p, dt, n, batch, reps)
        best = min(times.values())
        rows.append({"row": name, "op": op_name, "n": n, "batch": batch, "space": space,
                     "bo_evaluations": bo_evals,
                     "ms": {k: round(v, 5) for k, v in times.items()},
                     "e": {k: round(best / v, 4) for k, v in times.items() if k != "exhaustive"}})
    per_op = {}
    for o in kinds:
        rs = [r for r in rows if r["op"] == o]
        if not rs:
            continue
        per_op[o] = {k: round(bp.phi([r["e"][k] for r in rs]), 4) for k in ("model", "analytic", "learned")}
        per_op[o]["sizes"] = [r["n"] for r in rs]
        per_op[o]["bo_evaluations"] = [r["bo_evaluations"] for r in rs]
        per_op[o]["space"] = [r["space"] for r in rs]
    allrows = rows
    return {"phi": per_op,
            "phi_all": {k: round(bp.phi([r["e"][k] for r in allrows]), 4) for k in ("model", "analytic", "learned")}
            if allrows else None,
            "rows": rows, "exhaustive_evaluations": exh_evals, "reps": reps,
            "seconds": round(time.time() - t0, 1),
            "method": "each plan re-timed by bplg_time_plan (median of %d launches, library-owned buffers of the "
                      "row's shape); e = fastest of the four / plan; Phi = harmonic mean over sizes (Section VI); "
                      "model = BPLG_TUNE_MODEL (GB300 cost model, 0 evaluations), analytic = the paper's guideline "
                      "(0 evaluations), learned = the plans the timed step ran (Bayesian optimisation, budget 40)"
                      % reps}


def precision_quality(bp, torch, peak, reps: int = 10, check_rows: int = 32):
    """The precision configuration's FFT rows (N = 2^10, 2^12, 2^14, batch
    2^26 / N, seeded U[-1, 1] data): the float32 CUDA-core path against the
    tensor-core path with BF16 and FP16 split operands, forward transforms.
    Float32 runs its default plan (the GB300 cost model's); each tensor-core
    precision runs the fastest of its enumerated plans (median of `reps`
    launches each), whose error is checked on `check_rows` sampled signals
    against numpy's float64 FFT (relative L2 per signal; tolerance
    1e-5 log2 N)."""
    t0 = time.time()
    st = torch.cuda.current_stream()

    def timed(fn, r):
        for _ in range(2):
            fn()
        ev = []
        for _ in range(r):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            ev.append((e0, e1))
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in ev)

    out = {}
    for n in (1 << 10, 1 << 12, 1 << 14):
        batch = (1 << 26) // n
        z = si.fft_c64(batch, n, seed=si.CONFIG_SEEDS["precision"], stream=n)
        zd = torch.from_numpy(z.view(np.float32).reshape(-1)).cuda()
        od = torch.empty_like(zd)
        rows = np.unique(np.random.default_rng(5).integers(0, batch, check_rows))
        ref = np.fft.fft(z[rows].astype(np.complex128), axis=1)

        def err():
            X = od.view(-1, 2 * n)[torch.from_numpy(rows).cuda()].cpu().numpy().view(np.complex64)
            e = np.linalg.norm(X.astype(np.complex128) - ref, axis=1) / np.linalg.norm(ref, axis=1)
            return float("%.3e" % e.max())

        gb = 16 * n * batch / 1e9
        row = {"batch": batch, "tolerance": round(1e-5 * math.log2(n), 6)}
        ms = timed(lambda: bp.fft_batched(zd, od, n, batch, -1), reps)
        row["fp32"] = {"ms": round(ms, 5), "hbm_frac": round(gb / (ms * 1e-3) / peak, 4), "err_max": err()}
        plans = bp.enumerate_plans(bp.OP_FFT_TC, bp.F32, n)
        for name, prec in (("tc_bf16", bp.TC_BF16), ("tc_f16", bp.TC_F16)):
            best = None
            for p in plans:
                t = timed(lambda: bp.fft_tc_batched(zd, od, n, batch, -1, prec, plan=p), 3)
                if best is None or t < best[0]:
                    best = (t, p)
            p = best[1]
            ms = timed(lambda: bp.fft_tc_batched(zd, od, n, batch, -1, prec, plan=p), reps)
            row[name] = {"ms": round(ms, 5), "hbm_frac": round(gb / (ms * 1e-3) / peak, 4), "err_max": err(),
                         "plans_timed": len(plans),
                         "plan": {k: v for k, v in p.as_dict().items() if k in ("P", "L", "spb", "io")}}
        row["tc_over_fp32_speed"] = {k: round(row["fp32"]["ms"] / row[k]["ms"], 3) for k in ("tc_bf16", "tc_f16")}
        out[str(n)] = row
    out["seconds"] = round(time.time() - t0, 1)
    return out


def external_refs(torch, per_item, peak, reps: int = 20):
    """The vendor libraries on the same workloads and GPU, timed like the
    rows of the step (CUDA events on the current stream, median of `reps`
    launches after 3 warm-ups): cuFFT cufftPlanMany C2C for every FFT row,
    CUB's segmented InclusiveSumByKey for every scan row (and, for n = 8192,
    one InclusiveSum call per signal), cuSPARSE gtsv2StridedBatch for every
    tridiagonal row.  Context only: none of it is on the library's path.
    `ours_speedup` = the library's mean time / the reference's median time."""
    import ctypes
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_2310_16214_gb300", "_lib", "libbplg_extref.so"))
    vp, i64, szp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)
    lib.extref_scan_bykey.argtypes = [ctypes.c_int, vp, vp, i64, i64, vp, szp, vp]
    lib.extref_scan_each.argtypes = [ctypes.c_int, vp, vp, i64, i64, vp, szp, vp]
    lib.extref_fft_c2c.argtypes = [vp, vp, i64, i64, ctypes.c_int, vp]
    lib.extref_gtsv2.argtypes = [vp, vp, vp, vp, i64, i64, vp, szp, vp]
    st = torch.cuda.current_stream()
    sh = vp(st.cuda_stream)
    dev = torch.device("cuda", torch.cuda.current_device())

    def ok(rc, what):
        if rc != 0:
            raise RuntimeError("%s failed (%d)" % (what, rc))

    def timeit(fn, pre=None):
        for _ in range(3):
            if pre:
                pre()
            fn()
        evs = []
        for _ in range(reps):
            if pre:
                pre()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in evs)

    def entry(name, ms, elems, nbytes, rows):
        e = {"ms": round(ms, 5), "gelem_s": round(elems / (ms * 1e-3) / 1e9, 2),
             "hbm_frac": round(nbytes / (ms * 1e-3) / 1e9 / peak, 4)}
        if name in per_item:
            e["ours_speedup"] = round(ms / per_item[name], 3)
        rows[name] = e

    out = {"cufft": {}, "cub_scan": {}, "cusparse_gtsv2": {}}
    for n in FFT_SIZES:
        batch = FFT_TOTAL // n
        zin = torch.rand(2 * n * batch, device=dev) * 2 - 1
        zout = torch.empty_like(zin)
        for d, tag in ((-1, "fwd"), (1, "inv")):
            ms = timeit(lambda d=d: ok(lib.extref_fft_c2c(vp(zin.data_ptr()), vp(zout.data_ptr()), n, batch, d, sh),
                                       "cufft"))
            entry("fft_%s_%d" % (tag, n), ms, n * batch, 16 * n * batch, out["cufft"])
        del zin, zout
    for dname, dt, tdt in (("i32", 0, torch.int32), ("f32", 1, torch.float32)):
        for n in SCAN_SIZES:
            batch = SCAN_TOTAL // n
            xin = (torch.randint(-1000, 1001, (n * batch,), device=dev, dtype=torch.int32).to(tdt))
            xout = torch.empty_like(xin)
            need = ctypes.c_size_t(0)
            ok(lib.extref_scan_bykey(dt, vp(xin.data_ptr()), vp(xout.data_ptr()), n, batch, None, ctypes.byref(need),
                                     sh), "cub bykey size")
            tmp = torch.empty(max(1, need.value), dtype=torch.uint8, device=dev)
            ms = timeit(lambda: ok(lib.extref_scan_bykey(dt, vp(xin.data_ptr()), vp(xout.data_ptr()), n, batch,
                                                         vp(tmp.data_ptr()), ctypes.byref(need), sh), "cub bykey"))
            entry("scan_%s_%d" % (dname, n), ms, n * batch, 8 * n * batch, out["cub_scan"])
            if n == SCAN_SIZES[-1] and dname == "i32":
                each = ctypes.c_size_t(0)
                ok(lib.extref_scan_each(dt, vp(xin.data_ptr()), vp(xout.data_ptr()), n, batch, None,
                                        ctypes.byref(each), sh), "cub each size")
                tmp2 = torch.empty(max(1, each.value), dtype=torch.uint8, device=dev)
                ms = timeit(lambda: ok(lib.extref_scan_each(dt, vp(xin.data_ptr()), vp(xout.data_ptr()), n, batch,
                                                            vp(tmp2.data_ptr()), ctypes.byref(each), sh), "cub each"))
                e = {"ms": round(ms, 5), "gelem_s": round(n * batch / (ms * 1e-3) / 1e9, 2),
                     "calls": batch}
                if "scan_i32_%d" % n in per_item:
                    e["ours_speedup"] = round(ms / per_item["scan_i32_%d" % n], 3)
                out["cub_scan"]["scan_i32_%d_one_call_per_signal" % n] = e
            del xin, xout, tmp
    for n in TRI_SIZES:
        batch = TRI_TOTAL // n
        a = torch.rand(batch, n, device=dev) * 2 - 1
        c = torch.rand(batch, n, device=dev) * 2 - 1
        a[:, 0] = 0
        c[:, -1] = 0
        b = a.abs() + c.abs() + 1 + torch.rand(batch, n, device=dev)
        d = torch.rand(batch, n, device=dev) * 2 - 1
        x = torch.empty_like(d)
        need = ctypes.c_size_t(0)
        ok(lib.extref_gtsv2(vp(a.data_ptr()), vp(b.data_ptr()), vp(c.data_ptr()), vp(x.data_ptr()), n, batch, None,
                            ctypes.byref(need), sh), "gtsv2 size")
        buf = torch.empty(max(1, need.value), dtype=torch.uint8, device=dev)
        ms = timeit(lambda: ok(lib.extref_gtsv2(vp(a.data_ptr()), vp(b.data_ptr()), vp(c.data_ptr()),
                                                vp(x.data_ptr()), n, batch, vp(buf.data_ptr()), ctypes.byref(need),
                                                sh), "gtsv2"),
                    pre=lambda: x.copy_(d))
        entry("tridiag_%d" % n, ms, n * batch, 20 * n * batch, out["cusparse_gtsv2"])
        del a, b, c, d, x, buf
    return out


def measure_e2e(torch, wl, stream, args):
    """Same step through the public API with host buffers: every row's inputs
    are copied from pinned host memory, the row runs, and its outputs are
    copied back, all inside the timed region.  Copies in, compute and copies
    out go to three streams (the library calls take the stream): row k's
    outputs move out while row k+1's inputs move in (the link is full duplex),
    and row k+1's inputs may move in while row k runs; rows that share
    buffers are ordered by stream waits."""
    host_in, host_out = {}, {}
    h2d = d2h = 0
    for it in wl.items:
        host_in[it["name"]] = [x.cpu().pin_memory() for x in it["ins"]]
        host_out[it["name"]] = [torch.empty(x.shape, dtype=x.dtype).pin_memory() for x in it["outs"]]
        h2d += sum(x.numel() * x.element_size() for x in it["ins"])
        d2h += sum(x.numel() * x.element_size() for x in it["outs"])
    s_in = torch.cuda.Stream()
    s_out = torch.cuda.Stream()
    s_comp = torch.cuda.Stream()

    # rows that share a device buffer with an earlier row (the inverse FFT row
    # after the forward one of the same size) wait for it; every other row's
    # inputs move in while earlier rows run
    def ptrs(it):
        return {x.data_ptr() for x in it["ins"] + it["outs"]}

    items = wl.items
    shares_earlier = [any(ptrs(items[j]) & ptrs(items[k]) for j in range(k)) for k in range(len(items))]

    def step():
        for k, it in enumerate(items):
            if shares_earlier[k]:
                s_in.wait_stream(s_comp)  # earlier rows have finished with the shared buffers
            with torch.cuda.stream(s_in):
                for hx, dx in zip(host_in[it["name"]], it["ins"]):
                    dx.copy_(hx, non_blocking=True)
            s_comp.wait_stream(s_in)
            if k == 0 or shares_earlier[k]:
                # earlier output copies have left the shared buffers (at the
                # start of a step: every output copy of the previous step)
                s_comp.wait_stream(s_out)
            with torch.cuda.stream(s_comp):
                it["fn"]()  # the binding launches on the current stream
            s_out.wait_stream(s_comp)
            with torch.cuda.stream(s_out):
                for hx, dx in zip(host_out[it["name"]], it["outs"]):
                    hx.copy_(dx, non_blocking=True)
        s_in.wait_stream(s_comp)  # the next step's inputs overwrite this step's

    steps = max(1, min(args.steps, 5))
    step()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    s_in.wait_stream(stream)
    for _ in range(steps):
        step()
    stream.wait_stream(s_out)
    stream.wait_stream(s_comp)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    return {"value": round(wl.elems / (ms * 1e-3) / 1e9, 3), "unit": "Gelem/s", "ms_per_step": round(ms, 3),
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": steps,
            "copy_gb_s": round((h2d + d2h) / (ms * 1e-3) / 1e9, 1)}


# ----------------------------------------------------------- CPU oracle leg

def oracle_sample(sample_rows: int):
    """A bounded sample of every row of the step (inputs only)."""
    items = []
    for n in FFT_SIZES:
        rows = max(1, sample_rows * 64 // n)
        z = si.fft_c64(rows, n, stream=100 + n)
        items.append(("fft", -1, z))
        items.append(("fft", +1, z))
    for n in TRI_SIZES:
        rows = max(1, sample_rows * 64 // n)
        items.append(("thomas", 0, si.tridiag_f32(rows, n, stream=200 + n)[:4]))
    items.append(("thomas", 0, si.tridiag_f32(max(1, sample_rows // 16), REF_N,
                                              seed=si.CONFIG_SEEDS["precision"])[:4]))
    for n in SCAN_SIZES:
        rows = max(1, sample_rows * 256 // n)
        items.append(("scan_i32", 0, si.scan_i32(rows, n, stream=300 + n)))
        items.append(("scan_f32", 0, si.scan_f32(rows, n, stream=400 + n)))
    return items


def oracle_run(items):
    """Run the CPU oracle on a prepared sample; returns (elements, seconds)."""
    import oracle
    elems = 0
    t0 = time.perf_counter()
    for kind, arg, x in items:
        if kind == "fft":
            oracle.fft(x, arg)
            elems += x.size
        elif kind == "thomas":
            oracle.thomas(*x)
            elems += x[1].size
        elif kind == "scan_i32":
            oracle.scan_i32(x)
            elems += x.size
        else:
            oracle.scan_f32(x)
            elems += x.size
    return elems, time.perf_counter() - t0


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_run_parallel(items, cores: int):
    """The same oracle calls with every item's rows split into `cores`
    contiguous slices run by a thread pool (the oracle is C called through
    ctypes, which releases the interpreter lock during the call)."""
    from concurrent.futures import ThreadPoolExecutor
    chunks = []
    for kind, arg, x in items:
        rows = (x[0] if kind == "thomas" else x).shape[0]
        for c in range(cores):
            lo, hi = rows * c // cores, rows * (c + 1) // cores
            if hi > lo:
                chunks.append((kind, arg, tuple(a[lo:hi] for a in x) if kind == "thomas" else x[lo:hi]))
    with ThreadPoolExecutor(max_workers=cores) as ex:
        t0 = time.perf_counter()
        elems = sum(ex.map(lambda it: oracle_run([it])[0], chunks))
        secs = time.perf_counter() - t0
    return elems, secs


def cpu_baseline(args):
    """The oracle timed on the host: every core with the batch split across
    threads (the headline figure, `cores` = threads used), and one thread."""
    cores = host_cores()
    items = oracle_sample(args.cpu_rows)
    elems1, secs1 = oracle_run(items)
    itemsp = oracle_sample(2 * args.cpu_rows)
    elemsp, secsp = oracle_run_parallel(itemsp, cores)
    return {"value": round(elemsp / secsp / 1e9, 6), "unit": "Gelem/s", "cores": cores, "kind": "oracle",
            "single_thread": {"value": round(elems1 / secs1 / 1e9, 6), "cores": 1, "seconds": round(secs1, 2)},
            "sample": "%d elements across every row of the step (%d x 64 elements per FFT and tridiag size, "
                      "x 256 per scan size) split over %d threads, %.1f s; the single-thread figure uses half "
                      "that sample" % (elemsp, 2 * args.cpu_rows, cores, secsp)}


def run_reference(args):
    world, rank, local = dist_setup()
    if rank != 0:
        return
    # size each step's sample so the whole run stays near 90 s of CPU time
    cores = host_cores()
    cal_rows = 256
    _, cal_secs = oracle_run_parallel(oracle_sample(cal_rows), cores)
    per_row = max(cal_secs / cal_rows, 1e-9)
    rows = int(90.0 / max(1, args.steps + args.warmup) / per_row)
    items = oracle_sample(max(1, min(args.cpu_rows // 16, rows)))
    for _ in range(args.warmup):
        oracle_run_parallel(items, cores)
    elems = 0
    secs = 0.0
    for _ in range(args.steps):
        e, s = oracle_run_parallel(items, cores)
        elems += e
        secs += s
    value = elems / secs / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "Gelem/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * secs / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 (oracle)",
        "data": "synthetic (seeded SplitMix64, paper-shaped batches)",
        "config": {"workload": WORKLOAD, "sample": "bounded per-step sample of every row"},
        "cpu_baseline": {"value": round(value, 6), "unit": "Gelem/s", "kind": "oracle", "cores": cores,
                         "sample": "%d elements per step, every row of the step, batch split over %d threads"
                                   % (elems // max(1, args.steps), cores)},
        "e2e": {"value": round(value, 6), "unit": "Gelem/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def tune_report(args):
    """Tuned vs exhaustive (Section VI): for every op and size of the step, the
    analytical plan, the learned-cost-model (BO) plan and the exhaustive best,
    each re-timed back to back; e_i = t_best / t_plan and Phi per op."""
    import torch
    torch.cuda.set_device(0)
    import paper_2310_16214_gb300 as bp
    peak, _ = read_peaks()
    cases = [("fft", bp.OP_FFT, bp.F32, n, FFT_TOTAL // n, 16) for n in FFT_SIZES]
    cases += [("tridiag", bp.OP_TRIDIAG, bp.F32, n, TRI_TOTAL // n, 20) for n in TRI_SIZES]
    cases += [("tridiag_wm", bp.OP_TRIDIAG_WM, bp.F32, n, TRI_TOTAL // n, 20) for n in TRI_SIZES]
    cases += [("refined", bp.OP_TRIDIAG_REFINED, bp.F32, REF_N, REF_BATCH, 24)]
    cases += [("scan_i32", bp.OP_SCAN, bp.I32, n, SCAN_TOTAL // n, 8) for n in SCAN_SIZES]
    cases += [("scan_f32", bp.OP_SCAN, bp.F32, n, SCAN_TOTAL // n, 8) for n in SCAN_SIZES]
    if args.ops:
        keep = set(args.ops.split(","))
        cases = [c for c in cases if c[0] in keep]
    rows = []
    for name, op, dt, n, batch, bpe in cases:
        t0 = time.time()
        pa, _ = bp.tune_plan(op, dt, n, batch, bp.TUNE_ANALYTIC)
        pm, _ = bp.tune_plan(op, dt, n, batch, bp.TUNE_MODEL)
        pl, rl = bp.tune_plan(op, dt, n, batch, bp.TUNE_LEARNED, budget=args.bo_budget, seed=args.seed)
        pe, re_ = bp.tune_plan(op, dt, n, batch, bp.TUNE_EXHAUSTIVE)
        ta = bp.time_plan(pa, dt, n, batch, args.reps)
        tm = bp.time_plan(pm, dt, n, batch, args.reps)
        tl = bp.time_plan(pl, dt, n, batch, args.reps)
        te = bp.time_plan(pe, dt, n, batch, args.reps)
        best = min(ta, tm, tl, te)
        row = {"op": name, "n": n, "batch": batch, "space": re_.space_size,
               "analytic": {"plan": pa.as_dict(), "ms": round(ta, 5), "e": round(best / ta, 4)},
               "model": {"plan": pm.as_dict(), "ms": round(tm, 5), "e": round(best / tm, 4)},
               "learned": {"plan": pl.as_dict(), "ms": round(tl, 5), "e": round(best / tl, 4),
                           "evaluations": rl.evaluations},
               "exhaustive": {"plan": pe.as_dict(), "ms": round(te, 5), "evaluations": re_.evaluations},
               "best_gb_s": round(bpe * n * batch / (best * 1e-3) / 1e9, 1),
               "best_hbm_frac": round(bpe * n * batch / (best * 1e-3) / 1e9 / peak, 4),
               "seconds": round(time.time() - t0, 1)}
        rows.append(row)
        print(json.dumps(row), flush=True)
    ops = sorted(set(r["op"] for r in rows))
    summary = {}
    for o in ops:
        rs = [r for r in rows if r["op"] == o]
        summary[o] = {"phi_analytic": round(bp.phi([r["analytic"]["e"] for r in rs]), 4),
                      "phi_model": round(bp.phi([r["model"]["e"] for r in rs]), 4),
                      "phi_learned": round(bp.phi([r["learned"]["e"] for r in rs]), 4),
                      "bo_evaluations": [r["learned"]["evaluations"] for r in rs],
                      "space": [r["space"] for r in rs]}
    print(json.dumps({"tune_report": summary}))


def uneven_report(args):
    """The uneven batch (4096 int32 scans + 4096 FFTs + 4096 tridiagonal
    systems, sizes 2^U{5..13}) as one graph launch, against the same problems
    run as one batched launch per (operation, size) class with a plan tuned by
    the learned tuner for that class (budget 16), the launches back to back on
    one stream.  Median of `reps` runs each."""
    import torch
    torch.cuda.set_device(0)
    import paper_2310_16214_gb300 as bp
    dev = torch.device("cuda", 0)
    st = torch.cuda.current_stream()
    count = UNEVEN_COUNT
    seed = si.CONFIG_SEEDS["uneven"]
    ns = [int(v) for v in si.uneven_sizes(3 * count, seed)]
    wl = Workload(torch, bp, dev, rows=["uneven"], plans="query")
    graph = wl.items[0]["fn"]
    classes = {}
    for k, n in enumerate(ns):
        op = ("scan", "fft", "tridiag")[k // count]
        classes[(op, n)] = classes.get((op, n), 0) + 1
    launches = []
    for (op, n), b in sorted(classes.items()):
        if op == "scan":
            xin = torch.randint(-1000, 1001, (b * n,), device=dev, dtype=torch.int32)
            xout = torch.empty_like(xin)
            p, _ = bp.tune_plan(bp.OP_SCAN, bp.I32, n, b, bp.TUNE_LEARNED, budget=16, seed=args.seed)
            launches.append(lambda xin=xin, xout=xout, n=n, b=b, p=p: bp.scan_batched(xin, xout, n, b, dtype=bp.I32,
                                                                                     plan=p))
        elif op == "fft":
            zin = torch.rand(2 * b * n, device=dev) * 2 - 1
            zout = torch.empty_like(zin)
            p, _ = bp.tune_plan(bp.OP_FFT, bp.F32, n, b, bp.TUNE_LEARNED, budget=16, seed=args.seed)
            launches.append(lambda zin=zin, zout=zout, n=n, b=b, p=p: bp.fft_batched(zin, zout, n, b, -1, plan=p))
        else:
            a, bb, c, d, _ = si.tridiag_f32(b, n, stream=700 + n)
            ts = [torch.from_numpy(v).to(dev) for v in (a, bb, c, d)]
            x = torch.empty_like(ts[0])
            p, _ = bp.tune_plan(bp.OP_TRIDIAG, bp.F32, n, b, bp.TUNE_LEARNED, budget=16, seed=args.seed)
            launches.append(lambda ts=ts, x=x, n=n, b=b, p=p: bp.tridiag_batched(*ts, x, n, b, plan=p))

    def timeit(fn):
        for _ in range(3):
            fn()
        evs = []
        for _ in range(args.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in evs)

    def all_batched():
        for f in launches:
            f()

    g_ms = timeit(graph)
    b_ms = timeit(all_batched)
    row = {"uneven_report": {"items": 3 * count, "size_classes": len(classes), "graph_ms": round(g_ms, 5),
                             "batched_per_class_ms": round(b_ms, 5), "graph_speedup": round(b_ms / g_ms, 3),
                             "graph_gelem_s": round(sum(ns) / (g_ms * 1e-3) / 1e9, 2)}}
    print(json.dumps(row), flush=True)
    return row


def largefft_report(args):
    """FFTs above 16384 points (two kernels), N in {2^16, 2^18, 2^20, 2^22},
    2^24 / N signals: the GB300 cost model's, the analytical guideline's,
    the learned and the exhaustive plans over the joint knob space (split
    N1, columns per block, rows per block), each re-timed, Phi for the three
    tuners, and cuFFT on the same workload.  The
    algorithmic bytes are 16 per element, though the two passes move 32."""
    import ctypes
    import torch
    torch.cuda.set_device(0)
    import paper_2310_16214_gb300 as bp
    peak, _ = read_peaks()
    st = torch.cuda.current_stream()
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_2310_16214_gb300", "_lib", "libbplg_extref.so"))
    lib.extref_fft_c2c.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                   ctypes.c_void_p]

    def timeit(fn):
        for _ in range(3):
            fn()
        evs = []
        for _ in range(args.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in evs)

    rows, e_an, e_le, e_mo = [], [], [], []
    for logn in (16, 18, 20, 22):
        n = 1 << logn
        batch = (1 << 24) // n
        zin = torch.rand(2 * n * batch, device="cuda") * 2 - 1
        zout = torch.empty_like(zin)
        pa, _ = bp.tune_plan(bp.OP_FFT, bp.F32, n, batch, bp.TUNE_ANALYTIC)
        pm, _ = bp.tune_plan(bp.OP_FFT, bp.F32, n, batch, bp.TUNE_MODEL)
        pl, rl = bp.tune_plan(bp.OP_FFT, bp.F32, n, batch, bp.TUNE_LEARNED, budget=args.bo_budget, seed=args.seed)
        pe, re_ = bp.tune_plan(bp.OP_FFT, bp.F32, n, batch, bp.TUNE_EXHAUSTIVE)
        t = {k: timeit(lambda p=p: bp.fft_batched(zin, zout, n, batch, -1, plan=p))
             for k, p in (("model", pm), ("analytic", pa), ("learned", pl), ("exhaustive", pe))}
        best = min(t.values())
        tc = timeit(lambda: lib.extref_fft_c2c(ctypes.c_void_p(zin.data_ptr()), ctypes.c_void_p(zout.data_ptr()), n,
                                               batch, -1, ctypes.c_void_p(st.cuda_stream)))
        e_an.append(best / t["analytic"])
        e_mo.append(best / t["model"])
        e_le.append(best / t["learned"])
        row = {"n": n, "batch": batch, "space": re_.space_size, "bo_evaluations": rl.evaluations,
               "ms": {k: round(v, 5) for k, v in t.items()},
               "gelem_s": round(n * batch / (best * 1e-3) / 1e9, 1),
               "hbm_frac_algorithmic": round(16 * n * batch / (best * 1e-3) / 1e9 / peak, 4),
               "hbm_frac_two_pass": round(32 * n * batch / (best * 1e-3) / 1e9 / peak, 4),
               "cufft_ms": round(tc, 5), "ours_speedup_vs_cufft": round(tc / best, 3),
               "plans": {k: {"n1_log": p.n1_log, "spb": p.spb, "row_spb": p.row_spb}
                         for k, p in (("model", pm), ("analytic", pa), ("learned", pl), ("exhaustive", pe))}}
        rows.append(row)
        print(json.dumps(row), flush=True)
    phi = lambda es: round(len(es) / sum(1.0 / e for e in es), 4)
    print(json.dumps({"largefft_report": {"phi_model": phi(e_mo), "phi_analytic": phi(e_an), "phi_learned": phi(e_le)}}),
          flush=True)
    return rows


def nonpow2_report(args):
    """Lengths that are not powers of two, 2^24 elements per case: the padded
    scan (int32) and Wang-Mou solve on the next power of two against the
    power-of-two length just below, and FFTs against cuFFT (mixed radix for
    2^a 3^b 5^c up to 12288, Bluestein otherwise; cuFFT runs such lengths
    with its own mixed-radix or Bluestein kernels).  Every
    row reports the time, Gelem/s and the fraction of the measured copy
    bandwidth for the algorithmic bytes (scan 8, tridiag 20, FFT 16 per
    element)."""
    import ctypes
    import torch
    torch.cuda.set_device(0)
    import paper_2310_16214_gb300 as bp
    peak, _ = read_peaks()
    st = torch.cuda.current_stream()
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_2310_16214_gb300", "_lib", "libbplg_extref.so"))
    lib.extref_fft_c2c.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                   ctypes.c_void_p]

    def timeit(fn):
        for _ in range(3):
            fn()
        evs = []
        for _ in range(args.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in evs)

    def line(kind, n, batch, ms, bpe, extra=None):
        row = {"op": kind, "n": n, "batch": batch, "ms": round(ms, 5),
               "gelem_s": round(n * batch / (ms * 1e-3) / 1e9, 1),
               "hbm_frac": round(bpe * n * batch / (ms * 1e-3) / 1e9 / peak, 4)}
        row.update(extra or {})
        print(json.dumps(row), flush=True)
        return row

    rows = []
    total = 1 << 24
    for n in (1000, 1024, 5000, 4096):
        batch = total // n
        x = torch.randint(-1000, 1000, (n * batch,), dtype=torch.int32, device="cuda")
        y = torch.empty_like(x)
        rows.append(line("scan_i32", n, batch, timeit(lambda: bp.scan_batched(x, y, n, batch, dtype=bp.I32)), 8))
    for n in (1000, 1024, 3000, 2048):
        batch = total // n
        a, b, c, d, _ = si.tridiag_f32(batch, n, stream=950 + n)
        ts = [torch.from_numpy(v.reshape(-1)).cuda() for v in (a, b, c, d)]
        xo = torch.empty_like(ts[0])
        p = bp.query_plan(bp.OP_TRIDIAG_WM, bp.F32, 1 << (n - 1).bit_length(), batch)
        rows.append(line("tridiag_wm", n, batch, timeit(lambda: bp.tridiag_batched(*ts, xo, n, batch, plan=p)), 20,
                         {"plan_n": p.n}))
    for n in (1000, 3000, 6000, 10000, 375, 1001, 4095, 100003):
        batch = max(1, total // n)
        z = torch.rand(2 * n * batch, device="cuda") * 2 - 1
        zo = torch.empty_like(z)
        ms = timeit(lambda: bp.fft_batched(z, zo, n, batch, -1))
        tc = timeit(lambda: lib.extref_fft_c2c(ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(zo.data_ptr()), n, batch,
                                               -1, ctypes.c_void_p(st.cuda_stream)))
        v = n
        for f in (2, 3, 5):
            while v % f == 0:
                v //= f
        extra = {"cufft_ms": round(tc, 5), "ours_speedup_vs_cufft": round(tc / ms, 3)}
        if v == 1 and n <= 12288:
            kind = "fft_mixed_radix"
        else:
            kind = "fft_bluestein"
            extra["inner_M"] = 1 << (2 * n - 2).bit_length()
        rows.append(line(kind, n, batch, ms, 16, extra))
    return rows


def precision_report(args):
    """Precision configuration: FFT N in {2^10, 2^12, 2^14}, batch 2^26/N,
    tensor-core radix-16 stages with BF16 and FP16 split operands against
    the float32 CUDA-core Stockham path; error against numpy's float64 FFT
    on sampled signals (max and median relative L2) and the median time of
    `reps` launches (plans: learned tuner for each path)."""
    import torch
    torch.cuda.set_device(0)
    import paper_2310_16214_gb300 as bp
    peak, _ = read_peaks()
    out = []
    for n in (1 << 10, 1 << 12, 1 << 14):
        batch = (1 << 26) // n
        z = si.fft_c64(batch, n, seed=si.CONFIG_SEEDS["precision"], stream=n)
        zd = torch.from_numpy(z.view(np.float32).reshape(-1)).cuda()
        od = torch.empty_like(zd)
        rng = np.random.default_rng(3)
        rows = np.unique(rng.integers(0, batch, 64))
        ref = np.fft.fft(z[rows].astype(np.complex128), axis=1)
        st = torch.cuda.current_stream()
        paths = {
            "fp32": (bp.OP_FFT, lambda p: bp.fft_batched(zd, od, n, batch, -1, plan=p)),
            "tc_bf16": (bp.OP_FFT_TC, lambda p: bp.fft_tc_batched(zd, od, n, batch, -1, bp.TC_BF16, plan=p)),
            "tc_f16": (bp.OP_FFT_TC, lambda p: bp.fft_tc_batched(zd, od, n, batch, -1, bp.TC_F16, plan=p)),
        }
        row = {"n": n, "batch": batch}
        for name, (op, fn) in paths.items():
            p, rep = bp.tune_plan(op, bp.F32, n, batch, bp.TUNE_LEARNED, budget=40, seed=args.seed)
            for _ in range(3):
                fn(p)
            ts = []
            for _ in range(args.reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(st)
                fn(p)
                e1.record(st)
                ts.append((e0, e1))
            torch.cuda.synchronize()
            ms = statistics.median(a.elapsed_time(b) for a, b in ts)
            X = od.cpu().numpy().view(np.complex64).reshape(batch, n)[rows].astype(np.complex128)
            err = np.linalg.norm(X - ref, axis=1) / np.linalg.norm(ref, axis=1)
            row[name] = {"ms": round(ms, 5), "gelem_s": round(n * batch / (ms * 1e-3) / 1e9, 1),
                         "hbm_frac": round(16 * n * batch / (ms * 1e-3) / 1e9 / peak, 4),
                         "err_max": float("%.3e" % err.max()), "err_median": float("%.3e" % np.median(err)),
                         "tolerance": 1e-5 * math.log2(n), "plan": {k: v for k, v in p.as_dict().items()
                                                                    if k in ("P", "L", "spb", "smem_layout", "io")}}
        out.append(row)
        print(json.dumps(row), flush=True)
    return out


def case_run(args):
    """One FFT case on its own, for profiling: `--case fft` (bplg_fft_batched:
    any n, power of two, mixed radix or Bluestein) or `--case fft_tc`
    (bplg_fft_tc_batched with the first enumerated plan of `--io`, split
    `--precision`), forward, on 2^24 / n signals (or `--batch`) of U[-1, 1]
    data: `--warmup` untimed calls, then `--steps` timed ones; prints one
    JSON line with the mean time."""
    import torch
    torch.cuda.set_device(0)
    import paper_2310_16214_gb300 as bp
    n = args.n
    batch = args.batch or max(1, (1 << 24) // n)
    g = torch.Generator(device="cuda").manual_seed(args.seed)
    z = torch.rand(2 * n * batch, device="cuda", generator=g) * 2 - 1
    o = torch.empty_like(z)
    if args.case == "fft_tc":
        plan = [q for q in bp.enumerate_plans(bp.OP_FFT_TC, bp.F32, n) if q.io == args.io][0]
        fn = lambda: bp.fft_tc_batched(z, o, n, batch, -1, args.precision, plan=plan)
    else:
        plan = None
        fn = lambda: bp.fft_batched(z, o, n, batch, -1)
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(1, args.steps)
    print(json.dumps({"case": args.case, "n": n, "batch": batch, "ms": round(ms, 5),
                      "hbm_frac": round(16 * n * batch / (ms * 1e-3) / 1e9 / read_peaks()[0], 4),
                      "plan": plan.as_dict() if plan is not None else None, "device_status": bp.device_status()}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=float, default=1.0, help="fraction of the full batch sizes (testing only)")
    ap.add_argument("--cpu-rows", type=int, default=131072)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ext", action="store_true", help="skip the cuFFT / CUB / cuSPARSE references")
    ap.add_argument("--no-tuning", action="store_true",
                    help="skip the tuned-vs-exhaustive (Phi) measurement after the timed region")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the tensor-core vs float32 FFT comparison after the timed region")
    ap.add_argument("--tune-report", action="store_true", help="tuned vs exhaustive Phi report instead of the bench")
    ap.add_argument("--precision-report", action="store_true",
                    help="tensor-core (BF16/FP16 split) vs float32 FFT: error and time per N")
    ap.add_argument("--nonpow2-report", action="store_true",
                    help="scan / Wang-Mou / Bluestein FFT at lengths that are not powers of two")
    ap.add_argument("--largefft-report", action="store_true",
                    help="FFTs above 16384 points: tuners vs exhaustive (Phi) and cuFFT")
    ap.add_argument("--uneven-report", action="store_true",
                    help="the uneven batch's graph launch against one tuned batched launch per size class")
    ap.add_argument("--case", default="", choices=["", "fft", "fft_tc"],
                    help="time one FFT case (--n, --batch, --io, --precision) instead of the bench")
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--io", type=int, default=2)
    ap.add_argument("--precision", type=int, default=1, help="tensor-core split: 0 BF16, 1 FP16")
    ap.add_argument("--ops", default="", help="comma-separated ops for --tune-report")
    ap.add_argument("--reps", type=int, default=50)
    ap.add_argument("--bo-budget", type=int, default=40)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--rows", default="", help="comma-separated row names to run (default: every row)")
    ap.add_argument("--plans", default="learned", choices=["learned", "query"],
                    help="learned: Bayesian-optimisation tuning of every row before the timed region; "
                         "query: bplg_query_plan (cached tuned plan, else the analytical guideline)")
    ap.add_argument("--plan-json", default="", help='fixed plans: {"row": {"P": .., "spb": .., knob: ..}}')
    args = ap.parse_args()
    if args.tune_report:
        tune_report(args)
    elif args.precision_report:
        precision_report(args)
    elif args.uneven_report:
        uneven_report(args)
    elif args.nonpow2_report:
        nonpow2_report(args)
    elif args.case:
        case_run(args)
    elif args.largefft_report:
        largefft_report(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
