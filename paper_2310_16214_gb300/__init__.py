"""Python binding of the GB300 batched parallel-prefix library (libbplg.so).

Argument marshalling only: every computation runs in the library's CUDA
kernels, reached through the C ABI declared in ``include/bplg.h``.  The
functions keep the C names without the ``bplg_`` prefix and accept torch CUDA
tensors (PyTorch supplies device memory and streams) or raw integer device
pointers.  If the shared library has not been built, importing this package
raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libbplg.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_UNSUPPORTED_SIZE = -2
ERR_INVALID_PLAN = -3
ERR_CUDA = -4
ERR_TIMEOUT = -5
ERR_DEVICE_FLAG = -6
ERR_NO_DEVICE = -7

I32, F32 = 0, 1
OP_SCAN, OP_FFT, OP_TRIDIAG, OP_TRIDIAG_REFINED, OP_FFT_TC, OP_TRIDIAG_WM = 0, 1, 2, 3, 4, 5
PATTERN_KS, PATTERN_LF = 0, 1
TUNE_ANALYTIC, TUNE_LEARNED, TUNE_EXHAUSTIVE, TUNE_MODEL = 0, 1, 2, 3
TC_BF16, TC_F16 = 0, 1

EXPORTED = [
    "bplg_scan_batched", "bplg_fft_batched", "bplg_fft_tc_batched", "bplg_fft_batched_noalloc",
    "bplg_tridiag_batched",
    "bplg_tridiag_refined", "bplg_uneven_create", "bplg_uneven_launch", "bplg_uneven_units",
    "bplg_uneven_destroy",
    "bplg_arch_query", "bplg_arch_preset", "bplg_occupancy", "bplg_guideline_select", "bplg_phi",
    "bplg_enumerate_plans", "bplg_plan_resources", "bplg_tune_plan", "bplg_tune_plans_cost",
    "bplg_query_plan", "bplg_time_plan", "bplg_check_plan", "bplg_device_status", "bplg_last_error",
    "bplg_version", "bplg_set_online_tuning", "bplg_online_status",
]


class BplgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("bplg error %d: %s" % (code, msg))
        self.code = code


class Plan(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int32) for name in (
        "op", "n", "P", "L", "spb", "S", "radix", "shuffle", "pattern", "smem_layout", "smem_pad",
        "io", "cr_switch", "n1_log", "row_spb", "reserved")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}

    def __repr__(self):
        return "Plan(%s)" % ", ".join("%s=%d" % kv for kv in self.as_dict().items())

    def key(self):
        return tuple(self.as_dict().values())


class Arch(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int32) for name in (
        "max_warps_per_sm", "max_blocks_per_sm", "regs_per_sm", "reg_alloc_unit", "warp_alloc_granularity",
        "max_regs_per_thread", "smem_per_sm", "smem_alloc_unit", "max_smem_per_block",
        "smem_reserved_per_block", "max_threads_per_block", "num_sms")]


class Candidate(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int32) for name in ("S", "P", "L", "regs", "smem", "radix", "shuffle", "reserved")]


class TuneReport(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("space_size", ctypes.c_int32), ("evaluations", ctypes.c_int32),
                ("invalid", ctypes.c_int32), ("chosen_ms", ctypes.c_double), ("best_seen_ms", ctypes.c_double)]


class Item(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("n", ctypes.c_int32), ("dtype", ctypes.c_int32), ("dir", ctypes.c_int32),
                ("in_", ctypes.c_void_p * 4), ("out", ctypes.c_void_p)]


COST_FN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.POINTER(Plan), ctypes.c_void_p)


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            "libbplg.so is not built (%s); run `python -c \"import __graft_entry__ as g; g.build()\"`" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, I32_, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    PP = ctypes.POINTER(Plan)
    sig = {
        "bplg_scan_batched": ([I32_, P, P, I64, I64, PP, P], ctypes.c_int),
        "bplg_fft_batched": ([P, P, I64, I64, I32_, PP, P], ctypes.c_int),
        "bplg_fft_batched_noalloc": ([P, P, I64, I64, I32_, PP, P], ctypes.c_int),
        "bplg_fft_tc_batched": ([P, P, I64, I64, I32_, I32_, PP, P], ctypes.c_int),
        "bplg_tridiag_batched": ([P, P, P, P, P, I64, I64, PP, P], ctypes.c_int),
        "bplg_tridiag_refined": ([P, P, P, P, P, I64, I64, I32_, D, P, PP, P], ctypes.c_int),
        "bplg_uneven_create": ([ctypes.POINTER(Item), I64, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
        "bplg_uneven_launch": ([ctypes.c_void_p, P], ctypes.c_int),
        "bplg_uneven_units": ([ctypes.c_void_p, ctypes.POINTER(I32_)], ctypes.c_int),
        "bplg_uneven_destroy": ([ctypes.c_void_p], ctypes.c_int),
        "bplg_arch_query": ([I32_, ctypes.POINTER(Arch)], ctypes.c_int),
        "bplg_arch_preset": ([I32_, ctypes.POINTER(Arch)], ctypes.c_int),
        "bplg_occupancy": ([ctypes.POINTER(Arch), I32_, I32_, I32_, ctypes.POINTER(I32_), ctypes.POINTER(I32_)],
                           ctypes.c_int),
        "bplg_guideline_select": ([ctypes.POINTER(Arch), ctypes.POINTER(Candidate), I32_, I32_,
                                   ctypes.POINTER(I32_)], ctypes.c_int),
        "bplg_phi": ([ctypes.POINTER(D), I32_], D),
        "bplg_enumerate_plans": ([I32_, I32_, I64, PP, I32_, ctypes.POINTER(I32_)], ctypes.c_int),
        "bplg_plan_resources": ([PP, I32_, ctypes.POINTER(I32_), ctypes.POINTER(I32_), ctypes.POINTER(I32_)],
                                ctypes.c_int),
        "bplg_tune_plan": ([I32_, I32_, I64, I64, I32_, I32_, ctypes.c_uint64, PP, ctypes.POINTER(TuneReport)],
                           ctypes.c_int),
        "bplg_tune_plans_cost": ([PP, I32_, ctypes.POINTER(I32_), ctypes.POINTER(I32_), ctypes.POINTER(Arch), I32_,
                                  I32_, ctypes.c_uint64, COST_FN, P, ctypes.POINTER(I32_),
                                  ctypes.POINTER(TuneReport)], ctypes.c_int),
        "bplg_query_plan": ([I32_, I32_, I64, I64, PP], ctypes.c_int),
        "bplg_set_online_tuning": ([I32_, I32_, ctypes.c_uint64], ctypes.c_int),
        "bplg_online_status": ([I32_, I32_, I64, I64, ctypes.POINTER(I32_), ctypes.POINTER(I32_), PP], ctypes.c_int),
        "bplg_time_plan": ([PP, I32_, I64, I64, I32_, ctypes.POINTER(D)], ctypes.c_int),
        "bplg_check_plan": ([PP, I32_, I64], ctypes.c_int),
        "bplg_device_status": ([ctypes.POINTER(I32_), I32_], ctypes.c_int),
        "bplg_last_error": ([], ctypes.c_char_p),
        "bplg_version": ([], ctypes.c_int32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


lib = _load()


def last_error() -> str:
    m = lib.bplg_last_error()
    return m.decode() if m else ""


def _check(rc: int):
    if rc != OK:
        raise BplgError(rc, last_error())
    return rc


def _ptr(x) -> Optional[int]:
    """Device (or host) address of a torch tensor, or an int pointer, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _plan_ref(plan: Optional[Plan]):
    return ctypes.byref(plan) if plan is not None else None


def _need(name: str, t, nbytes: int) -> None:
    """A tensor argument must hold at least nbytes (the C ABI takes bare
    pointers and cannot check); raw integer pointers are the caller's."""
    if t is None or isinstance(t, int) or nbytes <= 0:
        return
    have = t.numel() * t.element_size()
    if have < nbytes:
        raise ValueError("%s holds %d bytes, the call needs %d" % (name, have, nbytes))


# ------------------------------------------------------------- compute calls

def scan_batched(inp, out, n: int, batch: int, dtype: Optional[int] = None, plan: Optional[Plan] = None,
                 stream=None) -> None:
    """Inclusive sum scan of [batch][n] int32 or float32 (see bplg_scan_batched)."""
    if dtype is None:
        import torch
        dtype = I32 if inp.dtype == torch.int32 else F32
    _need("in", inp, 4 * n * batch)
    _need("out", out, 4 * n * batch)
    _check(lib.bplg_scan_batched(dtype, _ptr(inp), _ptr(out), n, batch, _plan_ref(plan), _stream(stream)))


def fft_batched(inp, out, n: int, batch: int, direction: int = -1, plan: Optional[Plan] = None, stream=None) -> None:
    """Complex Stockham FFT of [batch][n] complex64 (see bplg_fft_batched)."""
    _need("in", inp, 8 * n * batch)
    _need("out", out, 8 * n * batch)
    _check(lib.bplg_fft_batched(_ptr(inp), _ptr(out), n, batch, direction, _plan_ref(plan), _stream(stream)))


def fft_tc_batched(inp, out, n: int, batch: int, direction: int = -1, precision: int = TC_BF16,
                   plan: Optional[Plan] = None, stream=None) -> None:
    """FFT with tensor-core radix-16 stages, split hi/lo operands (see bplg_fft_tc_batched)."""
    _need("in", inp, 8 * n * batch)
    _need("out", out, 8 * n * batch)
    _check(lib.bplg_fft_tc_batched(_ptr(inp), _ptr(out), n, batch, direction, precision, _plan_ref(plan),
                                   _stream(stream)))


def fft_batched_noalloc(inp, out, n: int, batch: int, direction: int = -1, plan: Optional[Plan] = None,
                        stream=None) -> None:
    """The FFT without any device allocation, n <= 4096 (see bplg_fft_batched_noalloc)."""
    _need("in", inp, 8 * n * batch)
    _need("out", out, 8 * n * batch)
    _check(lib.bplg_fft_batched_noalloc(_ptr(inp), _ptr(out), n, batch, direction, _plan_ref(plan),
                                        _stream(stream)))


def tridiag_batched(a, b, c, d, x, n: int, batch: int, plan: Optional[Plan] = None, stream=None) -> None:
    """Tridiagonal solve of [batch][n] float32 systems, CR/PCR or Wang-Mou by the plan's op
    (see bplg_tridiag_batched)."""
    for name, t in (("a", a), ("b", b), ("c", c), ("d", d), ("x", x)):
        _need(name, t, 4 * n * batch)
    _check(lib.bplg_tridiag_batched(_ptr(a), _ptr(b), _ptr(c), _ptr(d), _ptr(x), n, batch, _plan_ref(plan),
                                    _stream(stream)))


def tridiag_refined(a, b, c, d, x, n: int, batch: int, max_iter: int = 10, tol: float = 1e-14, iters=None,
                    plan: Optional[Plan] = None, stream=None) -> None:
    """Float64-residual refined solve; x is float64 (see bplg_tridiag_refined)."""
    for name, t in (("a", a), ("b", b), ("c", c), ("d", d)):
        _need(name, t, 4 * n * batch)
    _need("x", x, 8 * n * batch)
    _need("iters", iters, 4 * batch)
    _check(lib.bplg_tridiag_refined(_ptr(a), _ptr(b), _ptr(c), _ptr(d), _ptr(x), n, batch, max_iter, tol,
                                    _ptr(iters), _plan_ref(plan), _stream(stream)))


class UnevenBatch:
    """An uneven batch prepared once (bplg_uneven_create) and run with one
    graph launch per call (bplg_uneven_launch).  `items` is a list of dicts
    {op, n, in: [tensor, ...], out: tensor, dtype?, dir?}; the tensors must
    outlive the batch (they are kept referenced here)."""

    def __init__(self, items):
        arr = (Item * len(items))()
        self._keep = []
        for k, it in enumerate(items):
            e = arr[k]
            e.op, e.n = it["op"], it["n"]
            e.dtype = it.get("dtype", I32)
            e.dir = it.get("dir", -1)
            for q, t in enumerate(it["in"]):
                e.in_[q] = _ptr(t)
                self._keep.append(t)
            e.out = _ptr(it["out"])
            self._keep.append(it["out"])
        h = ctypes.c_void_p()
        _check(lib.bplg_uneven_create(arr, len(items), ctypes.byref(h)))
        self.handle = h

    def launch(self, stream=None) -> None:
        _check(lib.bplg_uneven_launch(self.handle, _stream(stream)))

    def units(self):
        u = (ctypes.c_int32 * 3)()
        _check(lib.bplg_uneven_units(self.handle, u))
        return tuple(u)

    def close(self) -> None:
        if self.handle:
            lib.bplg_uneven_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# -------------------------------------------------------------------- tuning

def arch_query(device: int = 0) -> Arch:
    a = Arch()
    _check(lib.bplg_arch_query(device, ctypes.byref(a)))
    return a


def arch_preset(which: int) -> Arch:
    """0 = GM20B (Jetson TX1), 1 = GB300."""
    a = Arch()
    _check(lib.bplg_arch_preset(which, ctypes.byref(a)))
    return a


def occupancy(arch: Arch, warps_per_block: int, regs_per_thread: int, smem_per_block: int):
    w, b = ctypes.c_int32(), ctypes.c_int32()
    _check(lib.bplg_occupancy(ctypes.byref(arch), warps_per_block, regs_per_thread, smem_per_block,
                              ctypes.byref(w), ctypes.byref(b)))
    return w.value, b.value


def guideline_select(arch: Arch, cands, radix_tunable: bool) -> int:
    arr = (Candidate * max(1, len(cands)))()
    for i, c in enumerate(cands):
        arr[i] = Candidate(c["S"], c["P"], c["L"], c["regs"], c["smem"], c.get("radix", 2), c.get("shuffle", 0), 0)
    out = ctypes.c_int32()
    _check(lib.bplg_guideline_select(ctypes.byref(arch), arr, len(cands), int(bool(radix_tunable)),
                                     ctypes.byref(out)))
    return out.value


def phi(efficiencies) -> float:
    arr = (ctypes.c_double * max(1, len(efficiencies)))(*efficiencies)
    return lib.bplg_phi(arr, len(efficiencies))


def enumerate_plans(op: int, dtype: int, n: int):
    count = ctypes.c_int32()
    _check(lib.bplg_enumerate_plans(op, dtype, n, None, 0, ctypes.byref(count)))
    arr = (Plan * max(1, count.value))()
    _check(lib.bplg_enumerate_plans(op, dtype, n, arr, count.value, ctypes.byref(count)))
    return [arr[i] for i in range(count.value)]


def plan_resources(plan: Plan, dtype: int = F32):
    r, s, t = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib.bplg_plan_resources(ctypes.byref(plan), dtype, ctypes.byref(r), ctypes.byref(s), ctypes.byref(t)))
    return r.value, s.value, t.value


def tune_plan(op: int, dtype: int, n: int, batch: int, method: int, budget: int = 0, seed: int = 0):
    p, rep = Plan(), TuneReport()
    _check(lib.bplg_tune_plan(op, dtype, n, batch, method, budget, seed, ctypes.byref(p), ctypes.byref(rep)))
    return p, rep


def tune_plans_cost(plans, cost, method: int, budget: int = 0, seed: int = 0, regs=None, smem=None, arch=None):
    """Search an explicit plan list with a Python objective cost(plan) -> ms."""
    k = len(plans)
    arr = (Plan * k)(*plans)
    regs_arr = (ctypes.c_int32 * k)(*regs) if regs is not None else None
    smem_arr = (ctypes.c_int32 * k)(*smem) if smem is not None else None
    cb = COST_FN(lambda pp, user: float(cost(pp.contents)))
    chosen, rep = ctypes.c_int32(), TuneReport()
    _check(lib.bplg_tune_plans_cost(arr, k, regs_arr, smem_arr, ctypes.byref(arch) if arch is not None else None,
                                    method, budget, seed, cb, None, ctypes.byref(chosen), ctypes.byref(rep)))
    return chosen.value, rep


def query_plan(op: int, dtype: int, n: int, batch: int) -> Plan:
    p = Plan()
    _check(lib.bplg_query_plan(op, dtype, n, batch, ctypes.byref(p)))
    return p


def set_online_tuning(enable: bool, budget: int = 40, seed: int = 0) -> None:
    """Spread the learned search over the calls themselves (see bplg_set_online_tuning)."""
    _check(lib.bplg_set_online_tuning(int(bool(enable)), budget, seed))


def online_status(op: int, dtype: int, n: int, batch: int):
    """(evaluations, finished, best plan so far or None) of the online search for one shape."""
    ev, fin, best = ctypes.c_int32(), ctypes.c_int32(), Plan()
    _check(lib.bplg_online_status(op, dtype, n, batch, ctypes.byref(ev), ctypes.byref(fin), ctypes.byref(best)))
    return ev.value, bool(fin.value), (best if best.op != 0 or best.n != 0 else None)


def time_plan(plan: Plan, dtype: int, n: int, batch: int, reps: int = 25) -> float:
    ms = ctypes.c_double()
    _check(lib.bplg_time_plan(ctypes.byref(plan), dtype, n, batch, reps, ctypes.byref(ms)))
    return ms.value


def check_plan(plan: Plan, dtype: int, n: int) -> int:
    return lib.bplg_check_plan(ctypes.byref(plan), dtype, n)


def device_status(reset: bool = False) -> int:
    """Device error word (0 = fine) recorded by the pipelined kernels."""
    f = ctypes.c_int32()
    _check(lib.bplg_device_status(ctypes.byref(f), int(reset)))
    return f.value


def version() -> int:
    return lib.bplg_version()


def make_plan(op: int, n: int, P: int, spb: int, **knobs) -> Plan:
    """Build a plan value; L and S follow from the knobs."""
    p = Plan()
    p.op, p.n, p.P, p.spb = op, n, P, spb
    p.L = spb * (n // P)
    p.radix = knobs.pop("radix", P if op in (OP_FFT, OP_FFT_TC) else 2)
    p.shuffle = knobs.pop("shuffle", 1 if op == OP_SCAN else 0)
    for k, v in knobs.items():
        setattr(p, k, v)
    return p
