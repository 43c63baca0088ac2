// Batched tridiagonal solver: cyclic reduction (CR, Fig. 1(a)) down to m
// equations, parallel cyclic reduction (PCR, Fig. 1(b)) on those m, then CR
// back substitution (Section III, "Tridiagonal system solvers"; knobs of
// Section V-A).  Equation i is a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i.
//
// A block holds `spb` systems of n = 2^logn equations in shared memory, one
// float4 (a, b, c, d) per equation, so every CR/PCR step reads or writes an
// equation with a single 16-byte access.  With smem_pad the row index i is
// stored at i + i/8 + i/64, which spreads the doubling strides of CR over the
// shared-memory banks.  Each system is served by tps = n/P threads.
//
// CR forward level with stride delta updates the equations i = 2 delta (u+1) - 1
// from their neighbours i -/+ delta:
//     k1 = a_i / b_{i-delta},  k2 = c_i / b_{i+delta}
//     a_i <- -a_{i-delta} k1,  c_i <- -c_{i+delta} k2
//     b_i <- b_i - c_{i-delta} k1 - a_{i+delta} k2
//     d_i <- d_i - d_{i-delta} k1 - d_{i+delta} k2
// until m = cr_switch equations remain, spaced n/m apart.  PCR then applies
// the same update to all m equations at doubling distances (in one warp with
// shuffles when `shuffle` is set, else through shared memory) until every
// equation is decoupled, x = d / b.  Back substitution walks the CR levels in
// reverse: x_i = (d_i - a_i x_{i-delta} - c_i x_{i+delta}) / b_i.  x overwrites
// d in place.  a_0 and c_{n-1} are never read (treated as 0).  Divisions use
// the hardware reciprocal (about 1 ulp), well inside the float32 tolerance.
//
// The refined variant keeps the original coefficients beside a working copy
// and x in float64; each iteration computes r = d - A x in float64 from the
// stored float32 coefficients, scales r by a power of two sigma so that
// max|r sigma| is in [1/2, 1), solves A e' = r sigma in float32 with the same
// CR/PCR code, and adds e = e' / sigma to x in float64.  A system stops when
// the correction just applied is below tol max|x|, or -- before solving --
// when its residual proves the error small: for a strictly diagonally
// dominant A, ||A^-1||_inf <= 1/delta with delta = min_i |b_i| - |a_i| - |c_i|
// (Varah's bound), so max|r| / delta <= tol max|x| bounds ||x - x*||.  With smem_layout 1 the
// coefficients are also cached as float64 in shared memory, so the residual
// needs no conversions (the float64 pipe is the bottleneck of this kernel).
#include <cmath>
#include <type_traits>

#include "device_util.cuh"
#include "fp_convert.cuh"
#include "internal.h"
#include "tma.cuh"
#include "tridiag_common.cuh"
#include "tridiag_wm.cuh"

namespace bplg {

// The block's tile of the four structure-of-arrays inputs, written as float4
// rows (a, b, c, d).  Row of system ss starts at rows + ss * row_stride.
template <int PAD>
__device__ __forceinline__ void tile_load_aos(const float *a, const float *b, const float *c, const float *d,
                                              float4 *rows, int row_stride, int logn, int count) {
    const int n = 1 << logn;
    if (logn >= 2) {  // a float4 of one array stays inside one system
        const int count4 = count >> 2;
        for (int q = threadIdx.x; q < count4; q += blockDim.x) {
            const float4 va = __ldcs(reinterpret_cast<const float4 *>(a) + q);
            const float4 vb = __ldcs(reinterpret_cast<const float4 *>(b) + q);
            const float4 vc = __ldcs(reinterpret_cast<const float4 *>(c) + q);
            const float4 vd = __ldcs(reinterpret_cast<const float4 *>(d) + q);
            const int e = q << 2;
            float4 *row = rows + (e >> logn) * row_stride;
            const int i = e & (n - 1);
            row[tpid<PAD>(i)] = make_float4(va.x, vb.x, vc.x, vd.x);
            row[tpid<PAD>(i + 1)] = make_float4(va.y, vb.y, vc.y, vd.y);
            row[tpid<PAD>(i + 2)] = make_float4(va.z, vb.z, vc.z, vd.z);
            row[tpid<PAD>(i + 3)] = make_float4(va.w, vb.w, vc.w, vd.w);
        }
    } else {
        for (int e = threadIdx.x; e < count; e += blockDim.x)
            rows[(e >> logn) * row_stride + tpid<PAD>(e & (n - 1))] =
                make_float4(__ldcs(a + e), __ldcs(b + e), __ldcs(c + e), __ldcs(d + e));
    }
}

// ---- compacted-level layout (smem_layout 1)
// Level l of cyclic reduction keeps its n >> l equations in an array of its
// own: the forward sweep reads equations 2v, 2v+1, 2v+2 of level l and writes
// the reduced equation v of level l+1, so every shared-memory access has
// stride 1 or 2 and one pad slot per 8 rows (cpid) makes them conflict-free.
// Level l, equation v is the original equation (v+1) 2^l - 1.  Every solved
// x goes to an original-order array (one pad per 32, xpid, conflict-free for
// the power-of-two strides of back substitution), from which back
// substitution reads the neighbours and the result is stored with 16-byte
// writes.
__device__ __forceinline__ int cpid(int i) { return i + (i >> 3); }
__device__ __forceinline__ int xpid(int i) { return i + (i >> 5); }
__host__ __device__ __forceinline__ int compact_level_size(int m) { return m + (m >> 3) + 1; }
__host__ __device__ __forceinline__ int compact_levels_elems(int n, int levels) {
    int e = 0;
    for (int l = 0; l <= levels; ++l) e += compact_level_size(n >> l);
    return e;
}
// bytes of one system: level rows (float4) then x (float), 16-byte multiple
__host__ __device__ __forceinline__ int compact_sys_bytes(int n, int levels) {
    const int xb = 4 * (n + (n >> 5) + 1);
    return 16 * compact_levels_elems(n, levels) + ((xb + 15) & ~15);
}

template <int SHUFFLE>
__device__ void cr_pcr_solve_compact(float4 *lv, float *X, int logn, int log_m, int t, int tps) {
    const int n = 1 << logn;
    const int levels = logn - log_m;
    // ---- forward: level l -> level l+1
    int off = 0;
    for (int ld = 0; ld < levels; ++ld) {
        const int ml = n >> ld;
        const int half = ml >> 1;
        const int off_next = off + compact_level_size(ml);
        const float4 *L = lv + off;
        float4 *N = lv + off_next;
        for (int v = t; v < half; v += tps) {
            const int i = 2 * v + 1;
            const float4 E = L[cpid(i)];
            const float4 Lq = L[cpid(i - 1)];
            const float k1 = E.x * frcp(Lq.y);
            float4 nw = make_float4(-Lq.x * k1, E.y - Lq.z * k1, 0.f, E.w - Lq.w * k1);
            if (i + 1 < ml) {
                const float4 Rq = L[cpid(i + 1)];
                const float k2 = E.z * frcp(Rq.y);
                nw.y -= Rq.x * k2;
                nw.w -= Rq.w * k2;
                nw.z = -Rq.z * k2;
            }
            N[cpid(v)] = nw;
        }
        off = off_next;
        __syncthreads();
    }
    // ---- PCR on the m contiguous equations of the top level
    float4 *Tp = lv + off;
    const int m = 1 << log_m;
    if constexpr (SHUFFLE) {
        if (t < 32) {
            const int width = tps < 32 ? tps : 32;
            const bool live = t < m;
            float4 q = live ? Tp[cpid(t)] : make_float4(0.f, 1.f, 0.f, 0.f);
            for (int sg = 1; sg < m; sg <<= 1) {
                const float am = __shfl_up_sync(kFullMask, q.x, sg, width);
                const float bm = __shfl_up_sync(kFullMask, q.y, sg, width);
                const float cm = __shfl_up_sync(kFullMask, q.z, sg, width);
                const float dm = __shfl_up_sync(kFullMask, q.w, sg, width);
                const float ap = __shfl_down_sync(kFullMask, q.x, sg, width);
                const float bp = __shfl_down_sync(kFullMask, q.y, sg, width);
                const float cp = __shfl_down_sync(kFullMask, q.z, sg, width);
                const float dp = __shfl_down_sync(kFullMask, q.w, sg, width);
                const bool hm = t >= sg;
                const bool hp = t + sg < m;
                const float k1 = hm ? q.x * frcp(bm) : 0.f;
                const float k2 = hp ? q.z * frcp(bp) : 0.f;
                float4 nw;
                nw.x = hm ? -am * k1 : 0.f;
                nw.z = hp ? -cp * k2 : 0.f;
                nw.y = q.y - (hm ? cm * k1 : 0.f) - (hp ? ap * k2 : 0.f);
                nw.w = q.w - (hm ? dm * k1 : 0.f) - (hp ? dp * k2 : 0.f);
                q = nw;
            }
            if (live) X[xpid(((t + 1) << levels) - 1)] = q.w * frcp(q.y);
        }
    } else {
        for (int sg = 1; sg < m; sg <<= 1) {
            float4 nw = make_float4(0.f, 1.f, 0.f, 0.f);
            if (t < m) {
                const float4 q = Tp[cpid(t)];
                nw = make_float4(0.f, q.y, 0.f, q.w);
                if (t >= sg) {
                    const float4 qm = Tp[cpid(t - sg)];
                    const float k1 = q.x * frcp(qm.y);
                    nw.x = -qm.x * k1;
                    nw.y -= qm.z * k1;
                    nw.w -= qm.w * k1;
                }
                if (t + sg < m) {
                    const float4 qp = Tp[cpid(t + sg)];
                    const float k2 = q.z * frcp(qp.y);
                    nw.z = -qp.z * k2;
                    nw.y -= qp.x * k2;
                    nw.w -= qp.w * k2;
                }
            }
            __syncthreads();
            if (t < m) Tp[cpid(t)] = nw;
            __syncthreads();
        }
        if (t < m) {
            const float4 q = Tp[cpid(t)];
            X[xpid(((t + 1) << levels) - 1)] = q.w * frcp(q.y);
        }
    }
    __syncthreads();
    // ---- back substitution: the even equations of level l.  Their
    // neighbours (the odd equations, original indices 2w 2^l - 1 and
    // (2w+2) 2^l - 1) were solved at higher levels; X holds every solved x.
    for (int ld = levels - 1; ld >= 0; --ld) {
        int o = 0;
        for (int l = 0; l < ld; ++l) o += compact_level_size(n >> l);
        const float4 *L = lv + o;
        const int half = (n >> ld) >> 1;
        for (int w = t; w < half; w += tps) {
            const float4 E = L[cpid(2 * w)];
            const float xl = w > 0 ? X[xpid(((2 * w) << ld) - 1)] : 0.f;
            const float xr = X[xpid(((2 * w + 2) << ld) - 1)];
            X[xpid(((2 * w + 1) << ld) - 1)] = (E.w - E.x * xl - E.z * xr) * frcp(E.y);
        }
        __syncthreads();
    }
}

// The block's tile of the four inputs written as level-0 rows of each
// system's compacted block (system ss at byte ss * sys_bytes).
__device__ __forceinline__ void tile_load_compact(const float *a, const float *b, const float *c, const float *d,
                                                  unsigned char *sm, int sys_bytes, int logn, int count) {
    const int n = 1 << logn;
    if (logn >= 2) {
        const int count4 = count >> 2;
        for (int q = threadIdx.x; q < count4; q += blockDim.x) {
            const float4 va = __ldcs(reinterpret_cast<const float4 *>(a) + q);
            const float4 vb = __ldcs(reinterpret_cast<const float4 *>(b) + q);
            const float4 vc = __ldcs(reinterpret_cast<const float4 *>(c) + q);
            const float4 vd = __ldcs(reinterpret_cast<const float4 *>(d) + q);
            const int e = q << 2;
            float4 *row = reinterpret_cast<float4 *>(sm + (e >> logn) * sys_bytes);
            const int i = e & (n - 1);
            row[cpid(i)] = make_float4(va.x, vb.x, vc.x, vd.x);
            row[cpid(i + 1)] = make_float4(va.y, vb.y, vc.y, vd.y);
            row[cpid(i + 2)] = make_float4(va.z, vb.z, vc.z, vd.z);
            row[cpid(i + 3)] = make_float4(va.w, vb.w, vc.w, vd.w);
        }
    } else {
        for (int e = threadIdx.x; e < count; e += blockDim.x)
            reinterpret_cast<float4 *>(sm + (e >> logn) * sys_bytes)[cpid(e & (n - 1))] =
                make_float4(__ldcs(a + e), __ldcs(b + e), __ldcs(c + e), __ldcs(d + e));
    }
}

__device__ __forceinline__ void tile_store_compact(float *x, unsigned char *sm, int sys_bytes, int x_off, int logn,
                                                   int count) {
    const int n = 1 << logn;
    if (logn >= 2) {
        const int count4 = count >> 2;
        for (int q = threadIdx.x; q < count4; q += blockDim.x) {
            const int e = q << 2;
            const float *X = reinterpret_cast<const float *>(sm + (e >> logn) * sys_bytes + x_off);
            const int i = e & (n - 1);
            __stcs(reinterpret_cast<float4 *>(x) + q,
                   make_float4(X[xpid(i)], X[xpid(i + 1)], X[xpid(i + 2)], X[xpid(i + 3)]));
        }
    } else {
        for (int e = threadIdx.x; e < count; e += blockDim.x)
            x[e] = reinterpret_cast<const float *>(sm + (e >> logn) * sys_bytes + x_off)[xpid(e & (n - 1))];
    }
}

template <int SHUFFLE>
__global__ void __launch_bounds__(1024)
    tridiag_compact_kernel(const float *a, const float *b, const float *c, const float *d, float *x, int logn,
                           int log_m, int log_tps, int spb, int64_t batch) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = 1 << logn;
    const int tps = 1 << log_tps;
    const int tid = threadIdx.x;
    const int s = tid >> log_tps;
    const int t = tid & (tps - 1);
    const int levels = logn - log_m;
    const int sys_bytes = compact_sys_bytes(n, levels);
    const int x_off = 16 * compact_levels_elems(n, levels);
    const int64_t sig0 = static_cast<int64_t>(blockIdx.x) * spb;
    const int64_t left = batch - sig0;
    const int nvalid = left < spb ? static_cast<int>(left) : spb;
    const int64_t off = sig0 * n;
    const int count = nvalid * n;
    unsigned char *mine = smem_raw + static_cast<size_t>(s) * sys_bytes;
    float4 *lv = reinterpret_cast<float4 *>(mine);
    float *X = reinterpret_cast<float *>(mine + x_off);

    tile_load_compact(a + off, b + off, c + off, d + off, smem_raw, sys_bytes, logn, count);
    __syncthreads();
    if (s >= nvalid) {
        for (int i = t; i < n; i += tps) lv[cpid(i)] = make_float4(0.f, 1.f, 0.f, 0.f);
    }
    if (t == 0) {
        lv[cpid(0)].x = 0.f;
        lv[cpid(n - 1)].z = 0.f;
    }
    __syncthreads();
    cr_pcr_solve_compact<SHUFFLE>(lv, X, logn, log_m, t, tps);
    tile_store_compact(x + off, smem_raw, sys_bytes, x_off, logn, count);
}

// ---- register cyclic reduction (smem_layout 2)
// Each thread owns P consecutive equations in registers and performs the
// first log2 P levels of cyclic reduction on them there.  At level l the
// updated equations are the local indices 2^(l+1) k - 1; all of them have
// their left neighbour in the thread, and all but the last (local P-1) their
// right one too.  The right neighbour of local P-1 is the next thread's local
// equation 2^l - 1 as it stands after level l-1, which that thread computes
// from its own data alone; so every thread first reduces everything except
// local P-1, publishes those log2 P "boundary" equations through shared
// memory (one barrier), and then reduces local P-1 with its neighbour's.
// Local P-1 is then the thread's equation of level log2 P: the n/P of them
// form a tridiagonal system on consecutive threads that the shared-memory
// CR/PCR code solves.  Back substitution of the register levels runs in
// registers again; only the previous thread's last x crosses threads.
template <int P, int PAD, int SHUFFLE, int MAXT>
__global__ void __launch_bounds__(MAXT)
    tridiag_reg_kernel(const float *ga, const float *gb, const float *gc, const float *gd, float *x, int logn,
                       int log_m, int log_tps, int spb, int64_t batch) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = 1 << logn;
    const int tps = 1 << log_tps;
    const int tid = threadIdx.x;
    const int s = tid >> log_tps;
    const int t = tid & (tps - 1);
    const int64_t sig0 = static_cast<int64_t>(blockIdx.x) * spb;
    const int64_t left = batch - sig0;
    const int nvalid = left < spb ? static_cast<int>(left) : spb;
    const int mstride = tstride<PAD>(tps);
    float4 *rows = reinterpret_cast<float4 *>(smem_raw) + s * mstride;
    float4 *bnd = reinterpret_cast<float4 *>(smem_raw) + spb * mstride;
    const int64_t g = (sig0 + s) * n + static_cast<int64_t>(t) * P;
    cr_register_system<P, PAD, SHUFFLE>(ga + g, gb + g, gc + g, gd + g, x + g, s < nvalid, log_m, log_tps, t, rows,
                                        bnd);
}

// Register-level CR fed by bulk asynchronous copies (smem_layout 2, io 1).
// A persistent block streams its tiles (spb systems) through one shared-
// memory slot: 4 copies per tile (a, b, c, d, each the tile's contiguous
// slice) complete on one mbarrier.  The slot is refilled as soon as every
// thread holds its run in registers, so the next tile's copy overlaps this
// tile's solve; one slot keeps the occupancy of the per-block kernel.  Each thread reads its P-run of the four arrays from the slot, the
// slot is refilled at once, and the solve is tridiag_reg_kernel's.  Waits
// are bounded: on timeout the block records an error, drains its own copies
// (bounded) and returns.
template <int P, int PAD, int SHUFFLE, int MAXT>
__global__ void __launch_bounds__(MAXT)
    tridiag_reg_tma_kernel(const float *ga, const float *gb, const float *gc, const float *gd, float *x, int logn,
                           int log_m, int log_tps, int spb, int64_t batch, int64_t ntiles) {
    constexpr int NS = 1;
    static_assert(P >= 4, "16-byte runs");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[NS];
    const int n = 1 << logn;
    const int tps = 1 << log_tps;
    const int tid = threadIdx.x;
    const int s = tid >> log_tps;
    const int t = tid & (tps - 1);
    const int slot_floats = spb * n;  // one array of one tile
    float *slots = reinterpret_cast<float *>(smem_raw);
    const int mstride = tstride<PAD>(tps);
    float4 *rows_base = reinterpret_cast<float4 *>(slots + NS * 4 * slot_floats);
    float4 *rows = rows_base + s * mstride;
    float4 *bnd = rows_base + spb * mstride;
    int issued[NS], consumed[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) issued[q] = consumed[q] = 0;

    auto issue = [&](int64_t tile, int q) {
        const int64_t sig0 = tile * spb;
        const int64_t left = batch - sig0;
        const int nv = left < spb ? static_cast<int>(left) : spb;
        const uint32_t bytes = static_cast<uint32_t>(nv) * static_cast<uint32_t>(n) * 4u;
        float *dst = slots + static_cast<size_t>(q) * 4 * slot_floats;
        mbar_arrive_expect_tx(&full[q], 4u * bytes);
        tma_load_1d(dst, ga + sig0 * n, bytes, &full[q]);
        tma_load_1d(dst + slot_floats, gb + sig0 * n, bytes, &full[q]);
        tma_load_1d(dst + 2 * slot_floats, gc + sig0 * n, bytes, &full[q]);
        tma_load_1d(dst + 3 * slot_floats, gd + sig0 * n, bytes, &full[q]);
        ++issued[q];
    };

    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NS; ++q) mbar_init(&full[q], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            const int64_t tile = blockIdx.x + static_cast<int64_t>(q) * gridDim.x;
            if (tile < ntiles) issue(tile, q);
        }
    }

    int k = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
        const int q = k % NS;
        const uint32_t parity = static_cast<uint32_t>(k / NS) & 1u;
        const int64_t sig0 = tile * spb;
        const int64_t left = batch - sig0;
        const int nvalid = left < spb ? static_cast<int>(left) : spb;
        const bool active = s < nvalid;
        const bool ok = __syncthreads_and(mbar_wait_bounded(&full[q], parity));
        if (!ok) {
            if (tid == 0) {  // drain this block's copies in flight, then leave
#pragma unroll
                for (int qq = 0; qq < NS; ++qq)
                    if (issued[qq] > consumed[qq]) mbar_wait_bounded(&full[qq], static_cast<uint32_t>(consumed[qq]) & 1u);
            }
            return;
        }
        if (tid == 0) ++consumed[q];
        float a[P], b[P], c[P], d[P];
        if (active) {
            const float *sl = slots + static_cast<size_t>(q) * 4 * slot_floats + s * n + t * P;
#pragma unroll
            for (int i = 0; i < P; i += 4) {
                const float4 va = *reinterpret_cast<const float4 *>(sl + i);
                const float4 vb = *reinterpret_cast<const float4 *>(sl + slot_floats + i);
                const float4 vc = *reinterpret_cast<const float4 *>(sl + 2 * slot_floats + i);
                const float4 vd = *reinterpret_cast<const float4 *>(sl + 3 * slot_floats + i);
                a[i] = va.x; a[i + 1] = va.y; a[i + 2] = va.z; a[i + 3] = va.w;
                b[i] = vb.x; b[i + 1] = vb.y; b[i + 2] = vb.z; b[i + 3] = vb.w;
                c[i] = vc.x; c[i + 1] = vc.y; c[i + 2] = vc.z; c[i + 3] = vc.w;
                d[i] = vd.x; d[i + 1] = vd.y; d[i + 2] = vd.z; d[i + 3] = vd.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < P; ++i) {
                a[i] = 0.f;
                b[i] = 1.f;
                c[i] = 0.f;
                d[i] = 0.f;
            }
        }
        __syncthreads();  // every run is in registers: refill the slot now
        const int64_t next = tile + static_cast<int64_t>(NS) * gridDim.x;
        if (tid == 0 && next < ntiles) {
            fence_proxy_async();
            issue(next, q);
        }
        if (t == 0) a[0] = 0.f;
        if (t == tps - 1) c[P - 1] = 0.f;
        cr_register_solve<P, PAD, SHUFFLE>(a, b, c, d, log_m, log_tps, t, rows, bnd);
        if (active) store_run<float, P>(x + (sig0 + s) * n + static_cast<int64_t>(t) * P, d);
    }
}

// Write the x column (the d components) of the block's rows to global memory.
template <int PAD>
__device__ __forceinline__ void tile_store_x(float *x, float4 *rows, int row_stride, int logn, int count) {
    const int n = 1 << logn;
    if (logn >= 2) {
        const int count4 = count >> 2;
        for (int q = threadIdx.x; q < count4; q += blockDim.x) {
            const int e = q << 2;
            float4 *row = rows + (e >> logn) * row_stride;
            const int i = e & (n - 1);
            __stcs(reinterpret_cast<float4 *>(x) + q,
                   make_float4(dcomp(row, tpid<PAD>(i)), dcomp(row, tpid<PAD>(i + 1)), dcomp(row, tpid<PAD>(i + 2)),
                               dcomp(row, tpid<PAD>(i + 3))));
        }
    } else {
        for (int e = threadIdx.x; e < count; e += blockDim.x)
            x[e] = dcomp(rows + (e >> logn) * row_stride, tpid<PAD>(e & (n - 1)));
    }
}

template <int PAD, int SHUFFLE>
__global__ void __launch_bounds__(1024)
    tridiag_kernel(const float *a, const float *b, const float *c, const float *d, float *x, int logn,
                   int log_m, int log_tps, int spb, int64_t batch) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *rows = reinterpret_cast<float4 *>(smem_raw);
    const int n = 1 << logn;
    const int tps = 1 << log_tps;
    const int tid = threadIdx.x;
    const int s = tid >> log_tps;
    const int t = tid & (tps - 1);
    const int64_t sig0 = static_cast<int64_t>(blockIdx.x) * spb;
    const int64_t left = batch - sig0;
    const int nvalid = left < spb ? static_cast<int>(left) : spb;
    const int stride = tstride<PAD>(n);
    const int64_t off = sig0 * n;
    const int count = nvalid * n;
    float4 *row = rows + s * stride;

    tile_load_aos<PAD>(a + off, b + off, c + off, d + off, rows, stride, logn, count);
    __syncthreads();
    if (s >= nvalid) {  // systems past the end of the batch: identity rows
        for (int i = t; i < n; i += tps) row[tpid<PAD>(i)] = make_float4(0.f, 1.f, 0.f, 0.f);
    }
    if (t == 0) {
        row[tpid<PAD>(0)].x = 0.f;
        row[tpid<PAD>(n - 1)].z = 0.f;
    }
    __syncthreads();
    cr_pcr_solve<PAD, SHUFFLE>(row, logn, log_m, t, tps);
    tile_store_x<PAD>(x + off, rows, stride, logn, count);
}

// Persistent, TMA-pipelined variant (io = 1).  Grid = the resident-block
// capacity; each block walks tiles of spb systems.  A ring of NS slots holds
// the tiles' four coefficient slices (one bulk asynchronous copy each, one
// mbarrier per slot), so the next tiles stream in while the current one is
// reduced.  The slot is unpacked into the padded float4 rows, refilled, and
// the rows are solved and stored as before.  Waits are bounded: on timeout
// the block records an error, drains its own copies (bounded) and returns.
template <int PAD, int SHUFFLE, int NS>
__global__ void __launch_bounds__(1024)
    tridiag_tma_kernel(const float *a, const float *b, const float *c, const float *d, float *x, int logn,
                       int log_m, int log_tps, int spb, int64_t batch, int64_t ntiles) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[NS];
    const int n = 1 << logn;
    const int tps = 1 << log_tps;
    const int tid = threadIdx.x;
    const int s = tid >> log_tps;
    const int t = tid & (tps - 1);
    const int stride = tstride<PAD>(n);
    const int tile_elems = spb * n;  // floats per coefficient slice (multiple of 4)
    float *slots = reinterpret_cast<float *>(smem_raw);
    float4 *rows = reinterpret_cast<float4 *>(slots + static_cast<size_t>(NS) * 4 * tile_elems);
    float4 *row = rows + s * stride;
    int issued[NS], consumed[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) issued[q] = consumed[q] = 0;

    auto issue = [&](int64_t tile, int q) {
        const int64_t sig0 = tile * spb;
        const int64_t left = batch - sig0;
        const int nv = left < spb ? static_cast<int>(left) : spb;
        const uint32_t bytes = static_cast<uint32_t>(nv) * static_cast<uint32_t>(n) * 4u;
        float *dst = slots + static_cast<size_t>(q) * 4 * tile_elems;
        const int64_t off = sig0 * n;
        mbar_arrive_expect_tx(&full[q], 4u * bytes);
        tma_load_1d(dst, a + off, bytes, &full[q]);
        tma_load_1d(dst + tile_elems, b + off, bytes, &full[q]);
        tma_load_1d(dst + 2 * tile_elems, c + off, bytes, &full[q]);
        tma_load_1d(dst + 3 * tile_elems, d + off, bytes, &full[q]);
        ++issued[q];
    };

    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NS; ++q) mbar_init(&full[q], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            const int64_t tile = blockIdx.x + static_cast<int64_t>(q) * gridDim.x;
            if (tile < ntiles) issue(tile, q);
        }
    }

    int k = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
        const int q = k % NS;
        const uint32_t parity = static_cast<uint32_t>(k / NS) & 1u;
        const int64_t sig0 = tile * spb;
        const int64_t left = batch - sig0;
        const int nvalid = left < spb ? static_cast<int>(left) : spb;
        const bool ok = __syncthreads_and(mbar_wait_bounded(&full[q], parity));
        if (!ok) {
            if (tid == 0) {
#pragma unroll
                for (int qq = 0; qq < NS; ++qq)
                    if (issued[qq] > consumed[qq]) mbar_wait_bounded(&full[qq], static_cast<uint32_t>(consumed[qq]) & 1u);
            }
            return;
        }
        if (tid == 0) ++consumed[q];
        // unpack the slot's slices into float4 rows (identity rows past the batch)
        const float *sa = slots + static_cast<size_t>(q) * 4 * tile_elems;
        if (s < nvalid) {
            const int so = s * n;
            for (int i = t; i < n; i += tps)
                row[tpid<PAD>(i)] = make_float4(i > 0 ? sa[so + i] : 0.f, sa[tile_elems + so + i],
                                                i < n - 1 ? sa[2 * tile_elems + so + i] : 0.f,
                                                sa[3 * tile_elems + so + i]);
        } else {
            for (int i = t; i < n; i += tps) row[tpid<PAD>(i)] = make_float4(0.f, 1.f, 0.f, 0.f);
        }
        __syncthreads();
        if (tid == 0) {
            const int64_t next = tile + static_cast<int64_t>(NS) * gridDim.x;
            if (next < ntiles) {
                fence_proxy_async();
                issue(next, q);
            }
        }
        cr_pcr_solve<PAD, SHUFFLE>(row, logn, log_m, t, tps);
        tile_store_x<PAD>(x + sig0 * n, rows, stride, logn, nvalid * n);
        __syncthreads();  // rows are rebuilt by the next tile
    }
}

constexpr int kTriTmaStages = 2;

// Maximum of v over the tps >= 32 threads of each system (every thread of the
// block calls; red holds one slot per warp).
__device__ __forceinline__ float system_max(float v, float *red, int wps) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFullMask, v, o));
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) red[warp] = v;
    __syncthreads();
    const int w0 = warp - (warp & (wps - 1));
    float r = red[w0];
    for (int k = 1; k < wps; ++k) r = fmaxf(r, red[w0 + k]);
    __syncthreads();
    return r;
}

// system_max with one barrier: red holds two sets of warp slots (64 floats)
// used alternately (ph toggles every call), so a call's writes never meet
// the previous call's reads -- every thread passes this call's barrier only
// after finishing the reads of the one before.
__device__ __forceinline__ float system_max1(float v, float *red, int wps, int &ph) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFullMask, v, o));
    float *slot = red + (ph & 1) * 32;
    ph ^= 1;
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) slot[warp] = v;
    __syncthreads();
    const int w0 = warp - (warp & (wps - 1));
    float r = slot[w0];
    for (int k = 1; k < wps; ++k) r = fmaxf(r, slot[w0 + k]);
    return r;
}

// Maximum of non-negative floats (magnitudes) over each system, with one
// barrier: their bit patterns order like the values, so each warp reduces
// them with one unsigned max.
__device__ __forceinline__ float system_max1_nonneg(float v, float *red, int wps, int &ph) {
    const unsigned w = __reduce_max_sync(kFullMask, __float_as_uint(v));
    float *slot = red + (ph & 1) * 32;
    ph ^= 1;
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) slot[warp] = __uint_as_float(w);
    __syncthreads();
    const int w0 = warp - (warp & (wps - 1));
    float r = slot[w0];
    for (int k = 1; k < wps; ++k) r = fmaxf(r, slot[w0 + k]);
    return r;
}

// The same two reductions for unsigned integers (high words of float64
// magnitudes, whose unsigned order is the order of the magnitudes).
__device__ __forceinline__ unsigned system_max_u(unsigned v, unsigned *red, int wps) {
    v = __reduce_max_sync(kFullMask, v);
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) red[warp] = v;
    __syncthreads();
    const int w0 = warp - (warp & (wps - 1));
    unsigned r = red[w0];
    for (int k = 1; k < wps; ++k) r = max(r, red[w0 + k]);
    __syncthreads();
    return r;
}
__device__ __forceinline__ unsigned system_max1_u(unsigned v, unsigned *red, int wps, int &ph) {
    v = __reduce_max_sync(kFullMask, v);
    unsigned *slot = red + (ph & 1) * 32;
    ph ^= 1;
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) slot[warp] = v;
    __syncthreads();
    const int w0 = warp - (warp & (wps - 1));
    unsigned r = slot[w0];
    for (int k = 1; k < wps; ++k) r = max(r, slot[w0 + k]);
    return r;
}

// Scale of a residual from the largest high word of its float64 entries
// (sign cleared): the exponent ex with max|r| in [2^(ex-1), 2^ex), clamped to
// [-120, 120] so that 2^ex and 2^-ex stay normal floats (0 for r = 0).
__device__ __forceinline__ int residual_exponent(unsigned rmax_hi) {
    const int ex = rmax_hi ? static_cast<int>(rmax_hi >> 20) - 1022 : 0;
    return ex < -120 ? -120 : (ex > 120 ? 120 : ex);
}

// Varah stopping threshold as a float64 high word: max|r| <= thr holds when
// the residual's largest high word plus one (an upper bound of max|r|) is at
// most this word.  rhs is 0 (never stop) or a normal float; the factor keeps
// the margin of the float32 tests.
__device__ __forceinline__ unsigned varah_hi(float rhs) {
    return fpc::hi_f64(fpc::widen_f32_normal(rhs * (1.0f - 1e-5f)));
}

// 2^e as float64 and float32, built from the exponent bits (exact).
__device__ __forceinline__ double pow2_f64(int e) {
    return __longlong_as_double(static_cast<long long>(1023 + e) << 52);
}
__device__ __forceinline__ float pow2_f32(int e) { return __int_as_float((127 + e) << 23); }

// The stopping tests run in float32 on float32 maxima: products of at most
// three float32 roundings, covered by the 1e-5 margins at their call sites.
// A right-hand side near the subnormal range would lose that accuracy, so
// below 2^-100 it becomes 0 and the test never stops the refinement.
__device__ __forceinline__ float stop_rhs(float v) { return v >= 7.8886091e-31f ? v : 0.f; }

// Shared memory of one system in the refined kernel, in bytes (16-byte
// multiple): the solver's working rows (strided rows, or compacted levels and
// the original-order x), original float32 rows, optional float64
// coefficients (a, b) and (c, d) pairs, and x in float64.
template <int PAD, int COEF64, int SOLVER>
__host__ __device__ __forceinline__ int refined_sys_bytes(int n, int levels) {
    const int work = SOLVER ? compact_sys_bytes(n, levels) : 16 * tstride<PAD>(n);
    return work + 16 * n + (COEF64 ? 32 * n : 0) + 8 * n + (n & 1) * 8;
}

template <int PAD, int SHUFFLE, int COEF64, int SOLVER>
__global__ void __launch_bounds__(1024)
    tridiag_refined_kernel(const float *a, const float *b, const float *c, const float *d, double *x,
                           int32_t *iters, int logn, int log_m, int log_tps, int spb, int64_t batch,
                           int max_iter, float tolf) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float red[32];
    __shared__ unsigned redu[32];
    __shared__ int done_sys[32];
    const int n = 1 << logn;
    const int tps = 1 << log_tps;
    const int wps = tps >> 5;
    const int tid = threadIdx.x;
    const int s = tid >> log_tps;
    const int t = tid & (tps - 1);
    const int64_t sig0 = static_cast<int64_t>(blockIdx.x) * spb;
    const int64_t left = batch - sig0;
    const int nvalid = left < spb ? static_cast<int>(left) : spb;
    const int stride = tstride<PAD>(n);
    const int64_t off = sig0 * n;
    const int count = nvalid * n;
    // per system: [work][orig rows][ab64][cd64][x64]
    const int levels = logn - log_m;
    const int work_bytes = SOLVER ? compact_sys_bytes(n, levels) : 16 * stride;
    unsigned char *base = smem_raw + static_cast<size_t>(s) * refined_sys_bytes<PAD, COEF64, SOLVER>(n, levels);
    float4 *w = reinterpret_cast<float4 *>(base);  // strided rows, or level-0 rows of the compacted layout
    float *Xc = reinterpret_cast<float *>(base + 16 * compact_levels_elems(n, levels));
    float4 *o = reinterpret_cast<float4 *>(base + work_bytes);
    double2 *ab = reinterpret_cast<double2 *>(base + work_bytes + 16 * n);
    double2 *cd = ab + n;
    double *xs = reinterpret_cast<double *>(base + work_bytes + 16 * n + (COEF64 ? 32 * n : 0));
    // working-row index of equation i and the solution of equation i
    auto widx = [&](int i) { return SOLVER ? cpid(i) : tpid<PAD>(i); };
    auto xsol = [&](int i) -> float & { return SOLVER ? Xc[xpid(i)] : dcomp(w, tpid<PAD>(i)); };
    auto solve = [&]() {
        if constexpr (SOLVER)
            cr_pcr_solve_compact<SHUFFLE>(w, Xc, logn, log_m, t, tps);
        else
            cr_pcr_solve<PAD, SHUFFLE>(w, logn, log_m, t, tps);
    };
    const bool valid = s < nvalid;

    // load this system's rows (each system reads its own contiguous slices)
    if (valid) {
        const int64_t so = off + static_cast<int64_t>(s) * n;
        for (int i = t; i < n; i += tps) {
            float4 q = make_float4(i > 0 ? __ldcs(a + so + i) : 0.f, __ldcs(b + so + i),
                                   i < n - 1 ? __ldcs(c + so + i) : 0.f, __ldcs(d + so + i));
            o[i] = q;
            w[widx(i)] = q;
            if constexpr (COEF64) {
                ab[i] = make_double2(fpc::widen_f32(q.x), fpc::widen_f32(q.y));
                cd[i] = make_double2(fpc::widen_f32(q.z), fpc::widen_f32(q.w));
            }
        }
    } else {
        for (int i = t; i < n; i += tps) {
            const float4 q = make_float4(0.f, 1.f, 0.f, 0.f);
            o[i] = q;
            w[widx(i)] = q;
            if constexpr (COEF64) {
                ab[i] = make_double2(0.0, 1.0);
                cd[i] = make_double2(0.0, 0.0);
            }
        }
    }
    if (t == 0) done_sys[s] = valid ? 0 : 1;
    __syncthreads();
    solve();
    // x0 = the float32 solution; max|x0| stands for max|x| in the stopping
    // test (the corrections change x by far less than its magnitude)
    float xmaxf = 0.f;
    for (int i = t; i < n; i += tps) {
        const float v = xsol(i);
        xs[i] = fpc::widen_f32(v);
        xmaxf = fmaxf(xmaxf, fabsf(v));
    }
    xmaxf = system_max(xmaxf, red, wps);
    // diagonal-dominance margin delta = min_i |b_i| - |a_i| - |c_i| (kept only
    // if positive, slightly shrunk for its float32 rounding): then
    // ||A^-1|| <= 1/delta and ||x - x*|| <= ||r|| / delta
    float dmin = 3.0e38f;
    for (int i = t; i < n; i += tps) {
        const float4 q = o[i];
        dmin = fminf(dmin, fabsf(q.y) - fabsf(q.x) - fabsf(q.z));
    }
    dmin = -system_max(-dmin, red, wps);
    const float dmarg = dmin > 0.f ? dmin * (1.0f - 1e-5f) : 0.f;
    // right-hand sides of the stopping tests below: 0 (never stop) unless
    // comfortably above the float32 subnormal range
    const unsigned varah_thr = varah_hi(stop_rhs(tolf * xmaxf * dmarg));
    const float corr_rhs = stop_rhs(tolf * xmaxf);

    int applied = 0;
    for (int k = 0;; ++k) {
        // residual r = d - A x in float64 from the stored float32 coefficients;
        // widening and narrowing are integer operations, so the FP64 pipe
        // carries only the three fused multiply-adds per equation.  The
        // float64 residual waits in the working row (its two halves in place
        // of c and d) until its largest entry is known; it is then scaled by
        // 2^-ex (max|r 2^-ex| in [1/2, 1)) as it is narrowed, so no entry is
        // lost to float32 underflow whatever the system's scale.
        unsigned rmax_hi = 0;
        for (int i = t; i < n; i += tps) {
            const float4 q = o[i];
            const double xl = i > 0 ? xs[i - 1] : 0.0;
            const double xr = i < n - 1 ? xs[i + 1] : 0.0;
            double r;
            if constexpr (COEF64) {
                const double2 p = ab[i], u = cd[i];
                r = fma(-p.x, xl, u.y);
                r = fma(-p.y, xs[i], r);
                r = fma(-u.x, xr, r);
            } else {
                r = fma(-fpc::widen_f32(q.x), xl, fpc::widen_f32(q.w));
                r = fma(-fpc::widen_f32(q.y), xs[i], r);
                r = fma(-fpc::widen_f32(q.z), xr, r);
            }
            const unsigned rh = fpc::hi_f64(r);
            rmax_hi = max(rmax_hi, rh & 0x7FFFFFFFu);
            w[widx(i)] = make_float4(q.x, q.y, __uint_as_float(rh), __uint_as_float(fpc::lo_f64(r)));
        }
        rmax_hi = system_max_u(rmax_hi, redu, wps);
        // the residual already bounds the error: stop before solving when
        // max|r| / delta <= tol max|x|
        if (t == 0 && rmax_hi + 1u <= varah_thr)
            done_sys[s] = 1;
        __syncthreads();
        {
            int all_done = 1;
            for (int q = 0; q < spb; ++q) all_done &= done_sys[q];
            __syncthreads();
            if (all_done || k == max_iter) break;
        }
        // the scaled residual 2^-ex r, narrowed, becomes the right-hand side
        const int ex = residual_exponent(rmax_hi);
        for (int i = t; i < n; i += tps) {
            const float4 row = w[widx(i)];
            const float rf = fpc::narrow_f64_ftz_pow2(
                fpc::f64_from_halves(__float_as_uint(row.z), __float_as_uint(row.w)), -ex);
            w[widx(i)] = make_float4(row.x, row.y, o[i].z, rf);
        }
        __syncthreads();
        solve();
        const bool was_done = done_sys[s] != 0 || rmax_hi == 0u;
        float emaxf = 0.f;
        for (int i = t; i < n; i += tps) {
            const float ep = xsol(i);
            if (!was_done) xs[i] += fpc::widen_f32_pow2(ep, ex);
            emaxf = fmaxf(emaxf, fabsf(ep));
        }
        emaxf = system_max(emaxf, red, wps);
        if (!was_done) ++applied;
        if (t == 0 && (was_done || emaxf * pow2_f32(ex) * (1.0f + 1e-5f) <= corr_rhs))
            done_sys[s] = 1;
        __syncthreads();
        int all_done = 1;
        for (int q = 0; q < spb; ++q) all_done &= done_sys[q];
        __syncthreads();
        if (all_done) break;
    }

    // store x (float64) and the correction counts
    if (valid) {
        double *xg = x + off + static_cast<int64_t>(s) * n;
        for (int i = 2 * t; i < n; i += 2 * tps)
            __stcs(reinterpret_cast<double2 *>(xg + i), make_double2(xs[i], xs[i + 1]));
        if (iters && t == 0) iters[sig0 + s] = applied;
    }
}

// Register-resident refinement (refined smem_layout 4, 5 and 6).  Each
// thread keeps its P equations' x in float64 and its working copy in
// registers; the float32 correction solves are the register-level CR (the
// middle system and boundary equations in shared memory), and the residual's
// neighbours across threads come from two float64 slots per thread.  The
// original coefficients, which every residual and every new working copy
// read, are kept (CO = 0, layout 4) as float32 registers; (CO = 1, layout 5)
// as float64 registers with float32 copies in shared memory; or (CO = 2,
// layout 6) as float32 rows in shared memory only, which frees 4P registers
// per thread for occupancy.  Shared-memory rows are stored [row][thread] so a
// warp's float4 accesses are contiguous.  The arithmetic is that of the
// shared-memory refinement.  With SOLVER = 1 (refined smem_layout 7, the
// coefficients as in layout 6) the float32 solves are the Wang-Mou divide
// and conquer (radix-2 merges, shuffles within a warp) instead of CR/PCR.
template <int P, int CO, int PAD, int SHUFFLE, int SOLVER, int LTPS = 0>
__device__ __forceinline__ void refined_reg_body(const float *ga, const float *gb, const float *gc, const float *gd,
                                                 double *x, int32_t *iters, int logn, int log_m, int log_tps_rt, int spb,
                                                 int64_t batch, int max_iter, float tolf) {
    // LTPS > 0: log2(threads per system) fixed at compile time (the
    // Wang-Mou merge stages then unroll with constant lanes and radices)
    const int log_tps = LTPS > 0 ? LTPS : log_tps_rt;
    constexpr int LP = (P >= 16) ? 4 : (P >= 8) ? 3 : (P >= 4) ? 2 : 1;
    constexpr int PF = CO == 0 ? P : 1;  // float32 coefficient registers (layout 4)
    constexpr int PD = CO == 1 ? P : 1;  // float64 coefficient registers (layout 5)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float red[64];
    __shared__ int done_sys[32];
    const int n = 1 << logn;
    const int tps = 1 << log_tps;
    const int wps = tps >> 5;
    const int tid = threadIdx.x;
    const int s = tid >> log_tps;
    const int t = tid & (tps - 1);
    const int64_t sig0 = static_cast<int64_t>(blockIdx.x) * spb;
    const int64_t left = batch - sig0;
    const int nvalid = left < spb ? static_cast<int>(left) : spb;
    const bool valid = s < nvalid;
    const int mstride = tstride<PAD>(tps);
    float4 *rows = reinterpret_cast<float4 *>(smem_raw) + s * mstride;
    float4 *bnd = reinterpret_cast<float4 *>(smem_raw) + spb * mstride;
    // Wang-Mou exchange buffer (4 float4 per thread) in place of rows + bnd
    float4 *wbuf = reinterpret_cast<float4 *>(smem_raw);
    double *xfirst = reinterpret_cast<double *>(reinterpret_cast<float4 *>(smem_raw) +
                                                (SOLVER ? 4 * blockDim.x : spb * mstride + blockDim.x * LP));
    double *xlast = xfirst + blockDim.x;
    // layouts 5 and 6: row i of this thread at ocoef[i * blockDim.x]
    float4 *ocoef = reinterpret_cast<float4 *>(xlast + blockDim.x) + tid;
    const int64_t g = (sig0 + s) * n + static_cast<int64_t>(t) * P;

    float la[P], lb[P], lc[P], ld[P];
    if (valid) {
        load_run<float, P>(ga + g, la);
        load_run<float, P>(gb + g, lb);
        load_run<float, P>(gc + g, lc);
        load_run<float, P>(gd + g, ld);
    } else {
#pragma unroll
        for (int i = 0; i < P; ++i) {
            la[i] = 0.f;
            lb[i] = 1.f;
            lc[i] = 0.f;
            ld[i] = 0.f;
        }
    }
    if (t == 0) la[0] = 0.f;
    if (t == tps - 1) lc[P - 1] = 0.f;
    float oa[PF], ob[PF], oc[PF], od[PF];
    double ca[PD], cb[PD], cc[PD], cd[PD];
    float dmin = 3.0e38f;
    // every coefficient of the block zero or normal (the usual case): the
    // residuals widen them with the short form
    // (on the magnitudes' bit patterns: the largest below infinity -- NaN and
    // inf fail -- and the smallest nonzero one at least 2^-126; a zero's
    // pattern minus one wraps to the largest and drops out of the minimum)
    unsigned amax = 0u, amin_m1 = 0xFFFFFFFFu;
#pragma unroll
    for (int i = 0; i < P; ++i) {
        const float v[4] = {la[i], lb[i], lc[i], ld[i]};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned m = __float_as_uint(v[k]) & 0x7FFFFFFFu;
            amax = max(amax, m);
            amin_m1 = min(amin_m1, m - 1u);
        }
    }
    const bool normal = amax < 0x7F800000u && amin_m1 >= 0x007FFFFFu;
    const bool fast = __syncthreads_and(normal) != 0;
#pragma unroll
    for (int i = 0; i < P; ++i) {
        dmin = fminf(dmin, fabsf(lb[i]) - fabsf(la[i]) - fabsf(lc[i]));
        if constexpr (CO == 1) {
            ca[i] = fpc::widen_f32(la[i]);
            cb[i] = fpc::widen_f32(lb[i]);
            cc[i] = fpc::widen_f32(lc[i]);
            cd[i] = fpc::widen_f32(ld[i]);
        }
        if constexpr (CO != 0) {
            ocoef[i * blockDim.x] = make_float4(la[i], lb[i], lc[i], ld[i]);
        } else {
            oa[i] = la[i];
            ob[i] = lb[i];
            oc[i] = lc[i];
            od[i] = ld[i];
        }
    }
    // la..ld become the working copy
    if (t == 0) done_sys[s] = valid ? 0 : 1;
    const bool single = spb == 1;  // (then the block's one system is valid)
    if constexpr (SOLVER == 1) {
        wm::wm_solve_inreg<P, 2, 1>(la, lb, lc, ld, log_tps, wbuf);
    } else {
        cr_register_solve<P, PAD, SHUFFLE>(la, lb, lc, ld, log_m, log_tps, t, rows, bnd);
    }
    double xs[P];
    float xmaxf = 0.f;
#pragma unroll
    for (int i = 0; i < P; ++i) {
        xs[i] = fpc::widen_f32(ld[i]);
        xmaxf = fmaxf(xmaxf, fabsf(ld[i]));
    }
    int ph = 0;
    xmaxf = system_max1_nonneg(xmaxf, red, wps, ph);
    // diagonal-dominance margin (see the shared-memory refinement)
    dmin = -system_max1(-dmin, red, wps, ph);
    const float dmarg = dmin > 0.f ? dmin * (1.0f - 1e-5f) : 0.f;
    // right-hand sides of the stopping tests below: 0 (never stop) unless
    // comfortably above the float32 subnormal range
    const unsigned varah_thr = varah_hi(stop_rhs(tolf * xmaxf * dmarg));
    const float corr_rhs = stop_rhs(tolf * xmaxf);
    unsigned *redu = reinterpret_cast<unsigned *>(red);  // shares red's two sets of warp slots (ph)

    int applied = 0;
    for (int k = 0;; ++k) {
        // neighbours of the first and last equation live in other threads
        xfirst[tid] = xs[0];
        xlast[tid] = xs[P - 1];
        __syncthreads();
        const double xl_nb = t > 0 ? xlast[tid - 1] : 0.0;
        const double xr_nb = t < tps - 1 ? xfirst[tid + 1] : 0.0;
        // residual r = d - A x in float64 from the stored float32 coefficients;
        // widening and narrowing are integer operations, so the FP64 pipe
        // carries only the three fused multiply-adds per equation.  The
        // float64 residual waits in ld (high half) and la (low half) until
        // its largest entry is known; it is then scaled by 2^-ex (max|r 2^-ex|
        // in [1/2, 1)) as it is narrowed, so no entry is lost to float32
        // underflow whatever the system's scale.
        unsigned rmax_hi = 0;
        auto residual = [&](auto fast_tag) {
            constexpr bool FAST = decltype(fast_tag)::value;
            auto widen = [](float f) { return FAST ? fpc::widen_f32_normal(f) : fpc::widen_f32(f); };
#pragma unroll
            for (int i = 0; i < P; ++i) {
                const double xl = i > 0 ? xs[i > 0 ? i - 1 : 0] : xl_nb;
                const double xr = i < P - 1 ? xs[i < P - 1 ? i + 1 : 0] : xr_nb;
                double r;
                if constexpr (CO == 1) {
                    r = fma(-ca[i], xl, cd[i]);
                    r = fma(-cb[i], xs[i], r);
                    r = fma(-cc[i], xr, r);
                } else if constexpr (CO == 2) {
                    const float4 q = ocoef[i * blockDim.x];
                    r = fma(-widen(q.x), xl, widen(q.w));
                    r = fma(-widen(q.y), xs[i], r);
                    r = fma(-widen(q.z), xr, r);
                } else {
                    r = fma(-widen(oa[i]), xl, widen(od[i]));
                    r = fma(-widen(ob[i]), xs[i], r);
                    r = fma(-widen(oc[i]), xr, r);
                }
                const unsigned rh = fpc::hi_f64(r);
                rmax_hi = max(rmax_hi, rh & 0x7FFFFFFFu);
                ld[i] = __uint_as_float(rh);
                la[i] = __uint_as_float(fpc::lo_f64(r));
            }
        };
        if (fast)
            residual(std::true_type{});
        else
            residual(std::false_type{});
        rmax_hi = system_max1_u(rmax_hi, redu, wps, ph);
        if (single) {
            // one system per block: every thread holds the same maxima and
            // takes the same decision, no flags or barriers needed
            if (rmax_hi + 1u <= varah_thr || k == max_iter) break;
        } else {
            if (t == 0 && rmax_hi + 1u <= varah_thr) done_sys[s] = 1;
            __syncthreads();
            int all_done = 1;
            for (int q = 0; q < spb; ++q) all_done &= done_sys[q];
            __syncthreads();
            if (all_done || k == max_iter) break;
        }
        // the scaled residual 2^-ex r, narrowed, becomes the right-hand side;
        // the correction solve's coefficients are read again only now, so
        // that just the residual's two halves stay live across the reduction
        const int ex = residual_exponent(rmax_hi);
#pragma unroll
        for (int i = 0; i < P; ++i) {
            ld[i] = fpc::narrow_f64_ftz_pow2(fpc::f64_from_halves(__float_as_uint(ld[i]), __float_as_uint(la[i])),
                                             -ex);
            if constexpr (CO == 0) {
                la[i] = oa[i];
                lb[i] = ob[i];
                lc[i] = oc[i];
            } else {
                const float4 q = ocoef[i * blockDim.x];
                la[i] = q.x;
                lb[i] = q.y;
                lc[i] = q.z;
            }
        }
        if constexpr (SOLVER == 1) {
            wm::wm_solve_inreg<P, 2, 1>(la, lb, lc, ld, log_tps, wbuf);
        } else {
            cr_register_solve<P, PAD, SHUFFLE>(la, lb, lc, ld, log_m, log_tps, t, rows, bnd);
        }
        const bool was_done = (!single && done_sys[s] != 0) || rmax_hi == 0u;
        float emaxf = 0.f;
#pragma unroll
        for (int i = 0; i < P; ++i) {
            if (!was_done) xs[i] += fpc::widen_f32_pow2(ld[i], ex);
            emaxf = fmaxf(emaxf, fabsf(ld[i]));
        }
        emaxf = system_max1_nonneg(emaxf, red, wps, ph);
        if (!was_done) ++applied;
        const bool small = was_done || emaxf * pow2_f32(ex) * (1.0f + 1e-5f) <= corr_rhs;
        if (single) {
            if (small) break;
        } else {
            if (t == 0 && small) done_sys[s] = 1;
            __syncthreads();
            int all_done = 1;
            for (int q = 0; q < spb; ++q) all_done &= done_sys[q];
            __syncthreads();
            if (all_done) break;
        }
    }
    if (valid) {
#pragma unroll
        for (int i = 0; i < P; i += 2) __stcs(reinterpret_cast<double2 *>(x + g + i), make_double2(xs[i], xs[i + 1]));
        if (iters && t == 0) iters[sig0 + s] = applied;
    }
}

template <int P, int CO, int PAD, int SHUFFLE, int MAXT, int SOLVER = 0>
__global__ void __launch_bounds__(MAXT)
    tridiag_refined_reg_kernel(const float *ga, const float *gb, const float *gc, const float *gd, double *x,
                               int32_t *iters, int logn, int log_m, int log_tps, int spb, int64_t batch,
                               int max_iter, float tolf) {
    refined_reg_body<P, CO, PAD, SHUFFLE, SOLVER>(ga, gb, gc, gd, x, iters, logn, log_m, log_tps, spb, batch,
                                                  max_iter, tolf);
}

// The same for blocks of at most MAXT threads with MINB of them resident per
// SM: the register cap that follows (65536 / (MAXT MINB)) trades a few
// spilled bytes for more resident warps.  Used by the Wang-Mou layout with
// P = 8 and blocks of up to 128 threads: 72 registers, 7 blocks per SM
// (0.256 ms at n = 1024, against 0.287 ms uncapped, 0.266 ms at 80 registers
// and 0.272 ms at 64; the P = 16 form capped at 96 registers spilled 432
// bytes and ran slower).  LTPS > 0 fixes log2(threads per system) at
// compile time.
template <int P, int CO, int PAD, int SHUFFLE, int MAXT, int SOLVER, int MINB, int LTPS = 0>
__global__ void __launch_bounds__(MAXT, MINB)
    tridiag_refined_reg_kernel_mb(const float *ga, const float *gb, const float *gc, const float *gd, double *x,
                                  int32_t *iters, int logn, int log_m, int log_tps, int spb, int64_t batch,
                                  int max_iter, float tolf) {
    refined_reg_body<P, CO, PAD, SHUFFLE, SOLVER, LTPS>(ga, gb, gc, gd, x, iters, logn, log_m, log_tps, spb, batch,
                                                        max_iter, tolf);
}

namespace {

// refined: layout bit 0 = float64 coefficient cache, bit 1 = compacted solver
template <int PAD, int SHUFFLE>
const void *tri_func_ps(bool refined, int layout, int io, int P, int threads, int log_tps) {
    if (refined && layout == 7) {  // Wang-Mou solves: unpadded, shuffle merges only
        if constexpr (PAD == 0 && SHUFFLE == 1) {
            switch (P) {
                case 2: return reinterpret_cast<const void *>(&tridiag_refined_reg_kernel<2, 2, 0, 1, 1024, 1>);
                case 4: return reinterpret_cast<const void *>(&tridiag_refined_reg_kernel<4, 2, 0, 1, 1024, 1>);
                case 8:
                    if (threads <= 128) {  // 72 registers: 7 blocks per SM
                        switch (log_tps) {  // merge stages unrolled at compile time
                            case 5: return reinterpret_cast<const void *>(&tridiag_refined_reg_kernel_mb<8, 2, 0, 1, 128, 1, 7, 5>);
                            case 6: return reinterpret_cast<const void *>(&tridiag_refined_reg_kernel_mb<8, 2, 0, 1, 128, 1, 7, 6>);
                            case 7: return reinterpret_cast<const void *>(&tridiag_refined_reg_kernel_mb<8, 2, 0, 1, 128, 1, 7, 7>);
                            default: break;
                        }
                        return reinterpret_cast<const void *>(&tridiag_refined_reg_kernel_mb<8, 2, 0, 1, 128, 1, 7>);
                    }
                    return reinterpret_cast<const void *>(&tridiag_refined_reg_kernel<8, 2, 0, 1, 512, 1>);
                case 16: return reinterpret_cast<const void *>(&tridiag_refined_reg_kernel<16, 2, 0, 1, 256, 1>);
                default: return nullptr;
            }
        }
        return nullptr;
    }
    if (refined && layout >= 4) {
        switch (layout * 32 + P) {
            case 4 * 32 + 2: return reinterpret_cast<const void *>(&tridiag_refined_reg_kernel<2, 0, PAD, SHUFFLE, 1024>);
            case 4 * 32 + 4: return reinterpret_cast<const void *>(&tridiag_refined_reg_kernel<4, 0, PAD, SHUFFLE, 512>);
            case 4 * 32 + 8: return reinterpret_cast<const void *>(&tridiag_refined_reg_kernel<8, 0, PAD, SHUFFLE, 256>);
            case 4 * 32 + 16: return reinterpret_cast<const void *>(&tridiag_refined_reg_kernel<16, 0, PAD, SHUFFLE, 256>);
            case 5 * 32 + 2: return reinterpret_cast<const void *>(&tridiag_refined_reg_kernel<2, 1, PAD, SHUFFLE, 512>);
            case 5 * 32 + 4: return reinterpret_cast<const void *>(&tridiag_refined_reg_kernel<4, 1, PAD, SHUFFLE, 512>);
            case 5 * 32 + 8: return reinterpret_cast<const void *>(&tridiag_refined_reg_kernel<8, 1, PAD, SHUFFLE, 256>);
            case 6 * 32 + 2: return reinterpret_cast<const void *>(&tridiag_refined_reg_kernel<2, 2, PAD, SHUFFLE, 1024>);
            case 6 * 32 + 4: return reinterpret_cast<const void *>(&tridiag_refined_reg_kernel<4, 2, PAD, SHUFFLE, 1024>);
            case 6 * 32 + 8: return reinterpret_cast<const void *>(&tridiag_refined_reg_kernel<8, 2, PAD, SHUFFLE, 512>);
            case 6 * 32 + 16: return reinterpret_cast<const void *>(&tridiag_refined_reg_kernel<16, 2, PAD, SHUFFLE, 256>);
            default: return nullptr;
        }
    }
    if (refined) {
        switch (layout) {
            case 0: return reinterpret_cast<const void *>(&tridiag_refined_kernel<PAD, SHUFFLE, 0, 0>);
            case 1: return reinterpret_cast<const void *>(&tridiag_refined_kernel<PAD, SHUFFLE, 1, 0>);
            case 2: return reinterpret_cast<const void *>(&tridiag_refined_kernel<PAD, SHUFFLE, 0, 1>);
            default: return reinterpret_cast<const void *>(&tridiag_refined_kernel<PAD, SHUFFLE, 1, 1>);
        }
    }
    if (layout == 1) return reinterpret_cast<const void *>(&tridiag_compact_kernel<SHUFFLE>);
    if (layout == 2 && io == 1) {
        switch (P) {
            case 4: return reinterpret_cast<const void *>(&tridiag_reg_tma_kernel<4, PAD, SHUFFLE, 1024>);
            case 8: return reinterpret_cast<const void *>(&tridiag_reg_tma_kernel<8, PAD, SHUFFLE, 512>);
            case 16: return reinterpret_cast<const void *>(&tridiag_reg_tma_kernel<16, PAD, SHUFFLE, 256>);
            default: return nullptr;
        }
    }
    if (layout == 2) {
        switch (P) {
            case 2: return reinterpret_cast<const void *>(&tridiag_reg_kernel<2, PAD, SHUFFLE, 1024>);
            case 4: return reinterpret_cast<const void *>(&tridiag_reg_kernel<4, PAD, SHUFFLE, 1024>);
            case 8: return reinterpret_cast<const void *>(&tridiag_reg_kernel<8, PAD, SHUFFLE, 512>);
            case 16: return reinterpret_cast<const void *>(&tridiag_reg_kernel<16, PAD, SHUFFLE, 256>);
            default: return nullptr;
        }
    }
    if (io == 1) return reinterpret_cast<const void *>(&tridiag_tma_kernel<PAD, SHUFFLE, kTriTmaStages>);
    return reinterpret_cast<const void *>(&tridiag_kernel<PAD, SHUFFLE>);
}

const void *tri_func(int pad, int shuffle, bool refined, int layout, int io, int P, int threads, int log_tps) {
    if (pad < 0 || pad > 1 || shuffle < 0 || shuffle > 1 || layout < 0 || layout > 7 || io < 0 || io > 1)
        return nullptr;
    if (!refined && layout == 1 && (pad != 1 || io != 0)) return nullptr;
    if (!refined && layout == 2 && io == 1 && P < 4) return nullptr;
    if (pad)
        return shuffle ? tri_func_ps<1, 1>(refined, layout, io, P, threads, log_tps)
                       : tri_func_ps<1, 0>(refined, layout, io, P, threads, log_tps);
    return shuffle ? tri_func_ps<0, 1>(refined, layout, io, P, threads, log_tps)
                   : tri_func_ps<0, 0>(refined, layout, io, P, threads, log_tps);
}

}  // namespace

int tridiag_smem_bytes(int pad, int64_t n, int spb, bool refined, int layout, int io, int log_m, int P) {
    const int ni = static_cast<int>(n);
    const int levels = ilog2(n) - log_m;
    if (!refined && layout == 1) return spb * compact_sys_bytes(ni, levels);
    if (!refined && layout == 2) {
        // middle rows per system + [threads][log2 P] boundary equations
        // (+ io 1: one slot of the tile's a, b, c, d)
        const int tps = ni / P;
        const int lp = ilog2(P);
        return (io == 1 ? 4 * spb * ni * 4 : 0) + spb * 16 * (pad ? tstride<1>(tps) : tps) + spb * tps * lp * 16;
    }
    if (!refined && io == 1) return kTriTmaStages * 16 * spb * ni + spb * 16 * (pad ? tstride<1>(ni) : ni);
    if (!refined) return spb * 16 * (pad ? tstride<1>(ni) : ni);
    if (layout == 7) {  // Wang-Mou exchanges + neighbour x slots + coefficient rows
        const int threads = spb * (ni / P);
        return threads * 64 + threads * 16 + spb * ni * 16;
    }
    if (layout >= 4) {  // register refinement: middle rows + boundary slots + neighbour x slots (+ rows)
        const int tps = ni / P;
        const int lp = ilog2(P);
        const int threads = spb * tps;
        return spb * 16 * (pad ? tstride<1>(tps) : tps) + threads * lp * 16 + threads * 16 +
               (layout >= 5 ? spb * ni * 16 : 0);
    }
    int per = 0;
    switch (layout) {
        case 0: per = pad ? refined_sys_bytes<1, 0, 0>(ni, levels) : refined_sys_bytes<0, 0, 0>(ni, levels); break;
        case 1: per = pad ? refined_sys_bytes<1, 1, 0>(ni, levels) : refined_sys_bytes<0, 1, 0>(ni, levels); break;
        case 2: per = refined_sys_bytes<1, 0, 1>(ni, levels); break;
        default: per = refined_sys_bytes<1, 1, 1>(ni, levels); break;
    }
    return spb * per;
}

bool tridiag_launch_info(const bplg_plan &p, int64_t n, int64_t batch, bool refined, Launch *out) {
    std::string why;
    bplg_plan q = p;
    if (!plan_structurally_valid(q, BPLG_F32, n, &why)) return false;
    const void *f = tri_func(p.smem_pad, p.shuffle, refined, p.smem_layout, refined ? 0 : p.io, p.P, p.L,
                             ilog2(n / p.P));
    if (!f) return false;
    out->func = f;
    out->threads = p.L;
    out->smem = tridiag_smem_bytes(p.smem_pad, n, p.spb, refined, p.smem_layout, refined ? 0 : p.io, ilog2(p.cr_switch),
                                   p.P);
    out->blocks = (batch + p.spb - 1) / p.spb;
    return true;
}

int tridiag_launch(const bplg_plan &p, const float *a, const float *b, const float *c,
                   const float *d, float *x, int64_t n, int64_t batch, cudaStream_t s) {
    Launch li;
    if (!tridiag_launch_info(p, n, batch, false, &li))
        return set_error(BPLG_ERR_INVALID_PLAN, "tridiag: plan has no kernel");
    int rc = check_grid(li.blocks, "tridiag");
    if (rc != BPLG_OK) return rc;
    rc = ensure_smem_attr(li.func, li.smem);
    if (rc != BPLG_OK) return rc;
    int logn = ilog2(n), log_m = ilog2(p.cr_switch), log_tps = ilog2(n / p.P), spb = p.spb;
    if (p.io == 1) {
        int64_t ntiles = li.blocks, grid = 0;
        rc = persistent_grid(li.func, li.threads, li.smem, ntiles, &grid);
        if (rc != BPLG_OK) return rc;
        void *args[] = {(void *)&a, (void *)&b, (void *)&c, (void *)&d, (void *)&x, &logn, &log_m, &log_tps, &spb, &batch,
                        &ntiles};
        cudaError_t e = cudaLaunchKernel(li.func, dim3(static_cast<unsigned>(grid)), dim3(li.threads), args,
                                         static_cast<size_t>(li.smem), s);
        return e == cudaSuccess ? BPLG_OK
                                : launch_error(e, "tridiag pipelined launch", li.func, grid, li.threads, li.smem);
    }
    void *args[] = {(void *)&a, (void *)&b, (void *)&c, (void *)&d, (void *)&x, &logn, &log_m, &log_tps, &spb, &batch};
    cudaError_t e = cudaLaunchKernel(li.func, dim3(static_cast<unsigned>(li.blocks)), dim3(li.threads), args,
                                     static_cast<size_t>(li.smem), s);
    return e == cudaSuccess ? BPLG_OK : cuda_error(e, "tridiag launch");
}

int tridiag_refined_launch(const bplg_plan &p, const float *a, const float *b, const float *c,
                           const float *d, double *x, int64_t n, int64_t batch, int max_iter,
                           double tol, int32_t *iters, cudaStream_t s) {
    // the kernels compare in float32 against a tolerance no larger than tol
    float tolf = static_cast<float>(tol);
    if (static_cast<double>(tolf) > tol) tolf = std::nextafter(tolf, 0.f);
    Launch li;
    if (!tridiag_launch_info(p, n, batch, true, &li))
        return set_error(BPLG_ERR_INVALID_PLAN, "tridiag refined: plan has no kernel");
    int rc = check_grid(li.blocks, "refined");
    if (rc != BPLG_OK) return rc;
    rc = ensure_smem_attr(li.func, li.smem);
    if (rc != BPLG_OK) return rc;
    int logn = ilog2(n), log_m = ilog2(p.cr_switch), log_tps = ilog2(n / p.P), spb = p.spb;
    void *args[] = {(void *)&a,    (void *)&b,  (void *)&c,     (void *)&d,  (void *)&x,      (void *)&iters, &logn,
                    &log_m,        &log_tps,    &spb,           &batch,      &max_iter,       &tolf};
    cudaError_t e = cudaLaunchKernel(li.func, dim3(static_cast<unsigned>(li.blocks)), dim3(li.threads), args,
                                     static_cast<size_t>(li.smem), s);
    return e == cudaSuccess ? BPLG_OK : cuda_error(e, "tridiag refined launch");
}

}  // namespace bplg

namespace bplg {

// Read (and optionally clear) the device error word of this file's kernels
// on the current device.
int tridiag_device_status(int *flag, bool reset) {
    int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_device_error, sizeof(int));
    if (e != cudaSuccess) return cuda_error(e, "device status");
    if (reset && v) {
        const int zero = 0;
        e = cudaMemcpyToSymbol(g_device_error, &zero, sizeof(int));
        if (e != cudaSuccess) return cuda_error(e, "device status reset");
    }
    *flag = v;
    return BPLG_OK;
}

}  // namespace bplg
