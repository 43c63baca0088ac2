// Device building blocks of cyclic reduction shared by the batched and the
// uneven-batch tridiagonal kernels: padded float4 rows, the in-place
// shared-memory CR/PCR solve, and the single CR elimination step.
#pragma once

#include <cuda_runtime.h>

#include "device_util.cuh"

namespace bplg {

template <int PAD>
__device__ __forceinline__ int tpid(int i) {
    return PAD ? i + (i >> 3) + (i >> 6) : i;
}

template <int PAD>
__host__ __device__ __forceinline__ int tstride(int n) {
    return PAD ? n + (n >> 3) + (n >> 6) + 1 : n;
}

__device__ __forceinline__ float frcp(float x) { return __fdividef(1.0f, x); }

__device__ __forceinline__ float &dcomp(float4 *row, int pi) { return reinterpret_cast<float *>(row + pi)[3]; }

// CR / PCR / back substitution on one system's rows.  Every thread of the
// block calls this (it synchronises the block); thread t in [0, tps) of each
// system does that system's share of the work.
template <int PAD, int SHUFFLE>
__device__ void cr_pcr_solve(float4 *row, int logn, int log_m, int t, int tps) {
    const int n = 1 << logn;
    const int levels = logn - log_m;
    // ---- cyclic reduction, forward
    for (int ld = 0; ld < levels; ++ld) {
        const int delta = 1 << ld;
        const int cnt = n >> (ld + 1);
        for (int u = t; u < cnt; u += tps) {
            const int i = ((u + 1) << (ld + 1)) - 1;
            const float4 E = row[tpid<PAD>(i)];
            const float4 Lq = row[tpid<PAD>(i - delta)];
            const float k1 = E.x * frcp(Lq.y);
            float4 nw = make_float4(-Lq.x * k1, E.y - Lq.z * k1, 0.f, E.w - Lq.w * k1);
            if (i + delta < n) {
                const float4 Rq = row[tpid<PAD>(i + delta)];
                const float k2 = E.z * frcp(Rq.y);
                nw.y -= Rq.x * k2;
                nw.w -= Rq.w * k2;
                nw.z = -Rq.z * k2;
            }
            row[tpid<PAD>(i)] = nw;
        }
        __syncthreads();
    }
    // ---- parallel cyclic reduction on the m remaining equations
    const int m = 1 << log_m;
    const int ls = levels;  // log2 of their spacing
    if constexpr (SHUFFLE) {
        if (t < 32) {  // the first warp (or segment) of each system
            const int width = tps < 32 ? tps : 32;
            const int jj = t;
            const bool live = jj < m;
            const int pi = tpid<PAD>(((jj + 1) << ls) - 1);
            float4 q = live ? row[pi] : make_float4(0.f, 1.f, 0.f, 0.f);
            for (int sg = 1; sg < m; sg <<= 1) {
                const float am = __shfl_up_sync(kFullMask, q.x, sg, width);
                const float bm = __shfl_up_sync(kFullMask, q.y, sg, width);
                const float cm = __shfl_up_sync(kFullMask, q.z, sg, width);
                const float dm = __shfl_up_sync(kFullMask, q.w, sg, width);
                const float ap = __shfl_down_sync(kFullMask, q.x, sg, width);
                const float bp = __shfl_down_sync(kFullMask, q.y, sg, width);
                const float cp = __shfl_down_sync(kFullMask, q.z, sg, width);
                const float dp = __shfl_down_sync(kFullMask, q.w, sg, width);
                const bool hm = jj >= sg;
                const bool hp = jj + sg < m;
                const float k1 = hm ? q.x * frcp(bm) : 0.f;
                const float k2 = hp ? q.z * frcp(bp) : 0.f;
                float4 nw;
                nw.x = hm ? -am * k1 : 0.f;
                nw.z = hp ? -cp * k2 : 0.f;
                nw.y = q.y - (hm ? cm * k1 : 0.f) - (hp ? ap * k2 : 0.f);
                nw.w = q.w - (hm ? dm * k1 : 0.f) - (hp ? dp * k2 : 0.f);
                q = nw;
            }
            if (live) dcomp(row, pi) = q.w * frcp(q.y);
        }
        __syncthreads();
    } else {
        const int jj = t;
        const int pi = tpid<PAD>(((jj + 1) << ls) - 1);
        for (int sg = 1; sg < m; sg <<= 1) {
            float4 nw = make_float4(0.f, 1.f, 0.f, 0.f);
            if (jj < m) {
                const float4 q = row[pi];
                nw = make_float4(0.f, q.y, 0.f, q.w);
                if (jj >= sg) {
                    const float4 qm = row[tpid<PAD>(((jj + 1 - sg) << ls) - 1)];
                    const float k1 = q.x * frcp(qm.y);
                    nw.x = -qm.x * k1;
                    nw.y -= qm.z * k1;
                    nw.w -= qm.w * k1;
                }
                if (jj + sg < m) {
                    const float4 qp = row[tpid<PAD>(((jj + 1 + sg) << ls) - 1)];
                    const float k2 = q.z * frcp(qp.y);
                    nw.z = -qp.z * k2;
                    nw.y -= qp.x * k2;
                    nw.w -= qp.w * k2;
                }
            }
            __syncthreads();
            if (jj < m) row[pi] = nw;
            __syncthreads();
        }
        if (jj < m) {
            const float4 q = row[pi];
            dcomp(row, pi) = q.w * frcp(q.y);
        }
        __syncthreads();
    }
    // ---- cyclic reduction, back substitution
    for (int ld = levels - 1; ld >= 0; --ld) {
        const int delta = 1 << ld;
        const int cnt = n >> (ld + 1);
        for (int u = t; u < cnt; u += tps) {
            const int i = (u << (ld + 1)) + delta - 1;
            const float4 E = row[tpid<PAD>(i)];
            const float xl = (i >= delta) ? dcomp(row, tpid<PAD>(i - delta)) : 0.f;
            const float xr = dcomp(row, tpid<PAD>(i + delta));
            dcomp(row, tpid<PAD>(i)) = (E.w - E.x * xl - E.z * xr) * frcp(E.y);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void cr_reduce(float &a, float &b, float &c, float &d, float la, float lb, float lc,
                                          float ld, float ra, float rb, float rc, float rd, bool has_right) {
    const float k1 = a * frcp(lb);
    float na = -la * k1, nb = b - lc * k1, nc = 0.f, nd = d - ld * k1;
    if (has_right) {
        const float k2 = c * frcp(rb);
        nb -= ra * k2;
        nd -= rd * k2;
        nc = -rc * k2;
    }
    a = na;
    b = nb;
    c = nc;
    d = nd;
}

// Register-level CR on the P equations a..d held by thread t of the tps
// threads serving one system (the register form of smem_layout 2).  rows is
// this system's padded middle system (tstride(tps) float4) and bnd the
// block's boundary-equation slots ([thread][log2 P] float4).  On return d
// holds x for the thread's equations (a, b, c are destroyed).  Every thread
// of the block calls it: two barriers plus those of the middle solve.
template <int P, int PAD, int SHUFFLE>
__device__ __forceinline__ void cr_register_solve(float (&a)[P], float (&b)[P], float (&c)[P], float (&d)[P],
                                                  int log_m, int log_tps, int t, float4 *rows, float4 *bnd) {
    constexpr int LP = (P >= 16) ? 4 : (P >= 8) ? 3 : (P >= 4) ? 2 : 1;
    const int tps = 1 << log_tps;
    const int tid = threadIdx.x;
    // phase A: every register level except local P-1; record the boundary
    // equations B_l = local 2^l - 1 as it stands after level l-1
    bnd[tid * LP + 0] = make_float4(a[0], b[0], c[0], d[0]);
#pragma unroll
    for (int l = 0; l < LP; ++l) {
        const int dl = 1 << l;
#pragma unroll
        for (int i = 2 * dl - 1; i < P - 1; i += 2 * dl)
            cr_reduce(a[i], b[i], c[i], d[i], a[i - dl], b[i - dl], c[i - dl], d[i - dl], a[i + dl], b[i + dl],
                      c[i + dl], d[i + dl], true);
        if (l + 1 < LP) {
            const int q = 2 * dl - 1;
            bnd[tid * LP + l + 1] = make_float4(a[q], b[q], c[q], d[q]);
        }
    }
    __syncthreads();
    // phase C: local P-1 through every register level with the next
    // thread's boundary equations
    const bool has_next = t < tps - 1;
#pragma unroll
    for (int l = 0; l < LP; ++l) {
        const int dl = 1 << l;
        float4 r = make_float4(0.f, 1.f, 0.f, 0.f);
        if (has_next) r = bnd[(tid + 1) * LP + l];
        cr_reduce(a[P - 1], b[P - 1], c[P - 1], d[P - 1], a[P - 1 - dl], b[P - 1 - dl], c[P - 1 - dl],
                  d[P - 1 - dl], r.x, r.y, r.z, r.w, has_next);
    }
    // the middle system: one equation per thread, consecutive
    rows[tpid<PAD>(t)] = make_float4(a[P - 1], b[P - 1], c[P - 1], d[P - 1]);
    __syncthreads();
    cr_pcr_solve<PAD, SHUFFLE>(rows, log_tps, log_m, t, tps);
    d[P - 1] = dcomp(rows, tpid<PAD>(t));  // x of local P-1 (d holds x from here on)
    const float xprev = t > 0 ? dcomp(rows, tpid<PAD>(t - 1)) : 0.f;
    // back substitution of the register levels
#pragma unroll
    for (int l = LP - 1; l >= 0; --l) {
        const int dl = 1 << l;
#pragma unroll
        for (int i = dl - 1; i < P - 1; i += 2 * dl) {
            const float xl = (i - dl >= 0) ? d[i - dl >= 0 ? i - dl : 0] : xprev;
            d[i] = (d[i] - a[i] * xl - c[i] * d[i + dl]) * frcp(b[i]);
        }
    }
}

// One system of the register-level CR read from and written to global
// memory: ga..gd, x point at this thread's P equations.
template <int P, int PAD, int SHUFFLE>
__device__ __forceinline__ void cr_register_system(const float *ga, const float *gb, const float *gc,
                                                   const float *gd, float *x, bool active, int log_m,
                                                   int log_tps, int t, float4 *rows, float4 *bnd) {
    const int tps = 1 << log_tps;
    float a[P], b[P], c[P], d[P];
    if (active) {
        load_run<float, P>(ga, a);
        load_run<float, P>(gb, b);
        load_run<float, P>(gc, c);
        load_run<float, P>(gd, d);
    } else {
#pragma unroll
        for (int i = 0; i < P; ++i) {
            a[i] = 0.f;
            b[i] = 1.f;
            c[i] = 0.f;
            d[i] = 0.f;
        }
    }
    if (t == 0) a[0] = 0.f;
    if (t == tps - 1) c[P - 1] = 0.f;
    cr_register_solve<P, PAD, SHUFFLE>(a, b, c, d, log_m, log_tps, t, rows, bnd);
    if (active) store_run<float, P>(x, d);
}

}  // namespace bplg
