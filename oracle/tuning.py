"""Plain-Python oracle for the tuning side: occupancy, the analytical
guideline, and the Phi performance-portability metric.

Test infrastructure only (see the package docstring).

* occupancy      -- Section IV-A: the active warps per SM W_SM and active
                    blocks per SM B_a, limited by the block cap B^max, the warp
                    cap W^max, the register file and shared memory; checked
                    against the GM20B table of Fig. 2(a).
* guideline      -- Section IV-A, the four-bullet tuning guideline, applied to
                    an explicit list of candidate configurations.
* phi            -- Section VI: Phi(a, C) = |C| / sum_i 1/e_i (harmonic mean of
                    the efficiencies e_i relative to the best observed).
* paper_space_*  -- the paper's search spaces on the Jetson TX1 (Section V:
                    TS, scan and FFT constraints) with the register and
                    shared-memory readings listed in each function, used to
                    reproduce the (S, P, L) tuples of Fig. 2(b)-(d).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence


@dataclass(frozen=True)
class Arch:
    """Per-SM resource limits that bound occupancy."""
    max_warps_per_sm: int          # W^max
    max_blocks_per_sm: int         # B^max
    regs_per_sm: int
    reg_alloc_unit: int            # registers per warp are rounded up to this
    warp_alloc_granularity: int    # warps limited by registers are floored to this
    max_regs_per_thread: int
    smem_per_sm: int
    smem_alloc_unit: int
    max_smem_per_block: int
    smem_reserved_per_block: int   # system use, added to every block
    max_threads_per_block: int


# Section II: GM20B (Jetson TX1) -- 64 warps and 32 blocks per SM, a 65536
# register file, 64 KB of shared memory per SM (48 KB per block), 1024
# threads per block.  Granularities are Maxwell's (256-register units, warps
# allocated in groups of 4, 256-byte shared-memory units).
TX1 = Arch(64, 32, 65536, 256, 4, 255, 65536, 256, 49152, 0, 1024)

# GB300 (sm_103): 64 warps and 32 blocks per SM, 65536 registers, 228 KB of
# shared memory per SM with 227 KB per block and 1 KB reserved per block.
GB300 = Arch(64, 32, 65536, 256, 4, 255, 233472, 128, 232448, 1024, 1024)


def _ceil_to(x: int, unit: int) -> int:
    return ((x + unit - 1) // unit) * unit


def occupancy(arch: Arch, warps_per_block: int, regs_per_thread: int, smem_per_block: int):
    """Return (W_SM, B_a) for one block shape; (0, 0) if it cannot launch."""
    w = warps_per_block
    if w <= 0 or w * 32 > arch.max_threads_per_block:
        return 0, 0
    if regs_per_thread > arch.max_regs_per_thread or smem_per_block > arch.max_smem_per_block:
        return 0, 0
    by_warps = arch.max_warps_per_sm // w
    if regs_per_thread > 0:
        regs_per_warp = _ceil_to(regs_per_thread * 32, arch.reg_alloc_unit)
        warps_by_regs = arch.regs_per_sm // regs_per_warp
        warps_by_regs -= warps_by_regs % arch.warp_alloc_granularity
        by_regs = warps_by_regs // w
    else:
        by_regs = arch.max_blocks_per_sm
    smem = smem_per_block + arch.smem_reserved_per_block
    if smem > 0:
        by_smem = arch.smem_per_sm // _ceil_to(smem, arch.smem_alloc_unit)
    else:
        by_smem = arch.max_blocks_per_sm
    b_a = min(arch.max_blocks_per_sm, by_warps, by_regs, by_smem)
    return b_a * w, b_a


@dataclass
class Candidate:
    """One configuration as the guideline sees it."""
    S: int
    P: int
    L: int
    regs: int
    smem: int
    radix: int = 2
    shuffle: int = 0
    tag: object = field(default=None, compare=False)

    @property
    def warps(self) -> int:
        return (self.L + 31) // 32


def guideline(arch: Arch, cands: Sequence[Candidate], radix_tunable: bool) -> Optional[int]:
    """Index of the configuration chosen by the Section IV-A guideline.

    Reading of the four bullets (every step keeps the candidate order as the
    final tie-break, so the first listed candidate wins a full tie):

    0. Premise (i), fewer high-latency communications: if some candidate that
       communicates by warp shuffles keeps W_SM/W^max >= 60 %, only shuffle
       candidates stay in the pool.
    4. Last bullet: for algorithms whose radix can grow (FFT, Wang & Mou),
       keep only the largest radix among the candidates with
       W_SM/W^max >= 60 %, even though that lowers B_a.
    1. Candidates with W_SM = W^max and B_a = B^max: take the largest P.
    2. Otherwise candidates with W_SM/W^max in [60 %, 100 %]: the largest B_a,
       then the largest P.
    3. Otherwise: the largest W_SM, then the largest P, then the largest B_a.
    """
    occ = []
    for c in cands:
        occ.append(occupancy(arch, c.warps, c.regs, c.smem))
    pool = [i for i, (w, b) in enumerate(occ) if b > 0]
    if not pool:
        return None
    wmax = arch.max_warps_per_sm

    def ratio(i):
        return occ[i][0] / wmax

    if any(cands[i].shuffle and ratio(i) >= 0.6 for i in pool):
        pool = [i for i in pool if cands[i].shuffle]
    if radix_tunable:
        good = [i for i in pool if ratio(i) >= 0.6]
        if good:
            rmax = max(cands[i].radix for i in good)
            pool = [i for i in pool if cands[i].radix == rmax]

    def first_best(ids, key):
        best = None
        for i in ids:
            if best is None or key(i) > key(best):
                best = i
        return best

    tier1 = [i for i in pool if occ[i][0] == wmax and occ[i][1] == arch.max_blocks_per_sm]
    if tier1:
        return first_best(tier1, lambda i: cands[i].P)
    tier2 = [i for i in pool if 0.6 <= ratio(i) <= 1.0]
    if tier2:
        return first_best(tier2, lambda i: (occ[i][1], cands[i].P))
    return first_best(pool, lambda i: (occ[i][0], cands[i].P, occ[i][1]))


def phi(efficiencies: Sequence[float]) -> float:
    """Phi(a, C) = |C| / sum_i 1/e_i (Section VI, harmonic mean)."""
    e = list(efficiencies)
    if not e or any(v <= 0 for v in e):
        return 0.0
    return len(e) / sum(1.0 / v for v in e)


# --------------------------------------------------------------------------
# The paper's search spaces on the TX1 (Section V)
# --------------------------------------------------------------------------

def _pow2_range(lo: int, hi: int) -> List[int]:
    out, v = [], lo
    while v <= hi:
        out.append(v)
        v *= 2
    return out


def paper_space_scan(N: int) -> List[Candidate]:
    """Scan (LF or KS), Section V-B: shuffle always on, P in {2..32}, L a power
    of two up to 1024, P*L a multiple of N (whole problems per block), 32
    shared-memory slots of 4 bytes per problem.  Register reading: 8*P (the
    paper keeps P <= 4 to stay within 32 registers)."""
    out = []
    for P in (2, 4, 8, 16, 32):
        for L in _pow2_range(32, 1024):
            if P * L < N or (P * L) % N:
                continue
            problems = P * L // N
            S = 32 * problems
            out.append(Candidate(S=S, P=P, L=L, regs=8 * P, smem=4 * S, radix=2, shuffle=1))
    return out


def paper_space_fft(N: int) -> List[Candidate]:
    """FFT, Section V-C: radix r = P in {2,4,8,16}, shared memory only, S = P*L
    holding whole problems, S <= 8192, real and imaginary parts exchanged in
    turn so 4 bytes per element are resident.  Register reading: 10*P (P = 4
    slightly exceeds 32 registers)."""
    out = []
    for P in (2, 4, 8, 16):
        if P > N:
            continue
        for L in _pow2_range(32, 1024):
            S = P * L
            if S < N or S % N or S > 8192:
                continue
            out.append(Candidate(S=S, P=P, L=L, regs=10 * P, smem=4 * S, radix=P, shuffle=0))
    return out


def paper_space_ts(N: int) -> List[Candidate]:
    """Tridiagonal CR / PCR, Section V-A: P in {2,4,8}, L in [32, 1024], S up to
    2048 equations of 16 bytes; shuffle only when N/P <= 32 and then S = 0,
    otherwise S = P*L.  Register reading: 10*P (P = 2 stays under 32, P = 4 is
    the 40-register case the paper quotes for WM)."""
    out = []
    for shuffle in (1, 0):
        for P in (2, 4, 8):
            if P > N:
                continue
            for L in _pow2_range(32, 1024):
                if P * L < N or (P * L) % N:
                    continue
                if shuffle:
                    if N // P > 32:
                        continue
                    S = 0
                else:
                    S = P * L
                    if S > 2048:
                        continue
                out.append(Candidate(S=S, P=P, L=L, regs=10 * P, smem=16 * S, radix=2, shuffle=shuffle))
    return out


def paper_tuple(op: str, N: int, arch: Arch = TX1):
    """(S, P, L) picked by the guideline for op in {'scan', 'fft', 'ts'}."""
    space = {"scan": paper_space_scan, "fft": paper_space_fft, "ts": paper_space_ts}[op](N)
    i = guideline(arch, space, radix_tunable=(op == "fft"))
    if i is None:
        return None
    c = space[i]
    return (c.S, c.P, c.L)
