// Device code of the Wang-Mou divide-and-conquer tridiagonal solver, shared
// by the batched kernel (tridiag_wm.cu), the uneven-batch kernel and the
// float32 solves of the refined kernel (layout 7).  The method and its
// mapping are described in tridiag_wm.cu.
#pragma once

#include <cuda_runtime.h>

#include "device_util.cuh"
#include "tridiag_common.cuh"

namespace bplg {
namespace wm {

// a + x X + y Y
struct Aff {
    float a, x, y;
};

// u = u.a + u.x XB + u.y YB with XB, YB themselves affine in (X, Y)
__device__ __forceinline__ Aff aff_compose(const Aff &u, const Aff &XB, const Aff &YB) {
    Aff r;
    r.a = fmaf(u.y, YB.a, fmaf(u.x, XB.a, u.a));
    r.x = fmaf(u.y, YB.x, u.x * XB.x);
    r.y = fmaf(u.y, YB.y, u.x * XB.y);
    return r;
}

// The outer neighbours of run g of an RS-run group, as affine functions of
// the group's outer neighbours (X, Y).  F[k] / L[k] describe the first /
// last unknown of run k in terms of run k's own neighbours.
template <int RS>
__device__ __forceinline__ void wm_outer(const Aff (&F)[RS], const Aff (&L)[RS], int g, Aff &XB, Aff &YB) {
    float p[RS - 1], q[RS - 1], sv[RS - 1], inv[RS - 1];
    p[0] = L[0].a;
    q[0] = L[0].x;
    sv[0] = L[0].y;
#pragma unroll
    for (int k = 1; k < RS - 1; ++k) {
        // u_{k-1} = p + q X + s v_{k-1} and v_{k-1} = F[k].a + F[k].x u_{k-1} + F[k].y v_k
        inv[k - 1] = frcp(1.f - sv[k - 1] * F[k].x);
        const float pp = fmaf(sv[k - 1], F[k].a, p[k - 1]) * inv[k - 1];
        const float qq = q[k - 1] * inv[k - 1];
        const float ss = sv[k - 1] * F[k].y * inv[k - 1];
        p[k] = fmaf(L[k].x, pp, L[k].a);
        q[k] = L[k].x * qq;
        sv[k] = fmaf(L[k].x, ss, L[k].y);
    }
    inv[RS - 2] = frcp(1.f - sv[RS - 2] * F[RS - 1].x);
    XB = Aff{0.f, 1.f, 0.f};
    YB = Aff{0.f, 0.f, 1.f};
    Aff vn = Aff{0.f, 0.f, 1.f};  // v_{k+1}, starting from Y
#pragma unroll
    for (int k = RS - 2; k >= 0; --k) {
        const Aff &f = F[k + 1];
        // v_k (1 - f.x s_k) = f.a + f.x (p_k + q_k X) + f.y v_{k+1}
        Aff v;
        v.a = fmaf(f.y, vn.a, fmaf(f.x, p[k], f.a)) * inv[k];
        v.x = fmaf(f.y, vn.x, f.x * q[k]) * inv[k];
        v.y = f.y * vn.y * inv[k];
        const Aff u = Aff{fmaf(sv[k], v.a, p[k]), fmaf(sv[k], v.x, q[k]), sv[k] * v.y};
        if (g == k) YB = v;      // run k's right neighbour is the first unknown of run k+1
        if (g == k + 1) XB = u;  // run k+1's left neighbour is the last unknown of run k
        vn = v;
    }
}

// One merge stage of radix RS over runs of S threads: gather the RS
// descriptors of this thread's group, then re-express the thread's own
// first/last descriptors in terms of the merged run's neighbours.
template <int RS>
__device__ __forceinline__ void wm_stage(Aff &Fo, Aff &Lo, int t, int log_s, bool by_shuffle, float4 *bf,
                                         float4 *bl) {
    const int S = 1 << log_s;
    const int G = S * RS;
    const int base = t & ~(G - 1);
    const int g = (t - base) >> log_s;
    Aff F[RS], L[RS];
    if (by_shuffle) {
        const int lbase = (threadIdx.x & 31) & ~(G - 1);
#pragma unroll
        for (int h = 0; h < RS; ++h) {
            const int sf = lbase + h * S, sl = sf + S - 1;
            F[h].a = __shfl_sync(kFullMask, Fo.a, sf);
            F[h].x = __shfl_sync(kFullMask, Fo.x, sf);
            F[h].y = __shfl_sync(kFullMask, Fo.y, sf);
            L[h].a = __shfl_sync(kFullMask, Lo.a, sl);
            L[h].x = __shfl_sync(kFullMask, Lo.x, sl);
            L[h].y = __shfl_sync(kFullMask, Lo.y, sl);
        }
    } else {
        const int tid = threadIdx.x;
        bf[tid] = make_float4(Fo.a, Fo.x, Fo.y, 0.f);
        bl[tid] = make_float4(Lo.a, Lo.x, Lo.y, 0.f);
        __syncthreads();
        const int sys0 = tid - t;  // this system's first thread in the block
#pragma unroll
        for (int h = 0; h < RS; ++h) {
            const float4 f = bf[sys0 + base + h * S];
            const float4 l = bl[sys0 + base + h * S + S - 1];
            F[h] = Aff{f.x, f.y, f.z};
            L[h] = Aff{l.x, l.y, l.z};
        }
    }
    Aff XB, YB;
    wm_outer<RS>(F, L, g, XB, YB);
    Fo = aff_compose(Fo, XB, YB);
    Lo = aff_compose(Lo, XB, YB);
}

// Shared memory of a block: two parities x (first, last) descriptors x one
// float4 per thread, unless every exchange is a warp shuffle.
__host__ __device__ __forceinline__ bool wm_warp_only(int shuffle, int64_t tps) { return shuffle && tps <= 32; }

// One system (or, with several systems per block, each of them) solved by
// the threads that serve it, from this thread's P equations in registers
// (identity rows where `active` is false).  a..c are destroyed and d ends
// holding the thread's P unknowns.  buf is the block's shared memory (4
// float4 per thread) unless every exchange is a warp shuffle.  Every thread
// of the block calls it.
template <int P, int R, int SHUFFLE>
__device__ __forceinline__ void wm_solve_inreg(float (&a)[P], float (&b)[P], float (&c)[P], float (&d)[P],
                                               int log_tps, float4 *buf) {
    const int tps = 1 << log_tps;
    const int tid = threadIdx.x;
    const int t = tid & (tps - 1);
    if (t == 0) a[0] = 0.f;
    if (t == tps - 1) c[P - 1] = 0.f;

    // (1) the thread's run: Thomas forward elimination for three right-hand
    // sides, then back substitution
    float cp[P], al[P], be[P], gm[P];
    {
        float inv = frcp(b[0]);
        cp[0] = c[0] * inv;
        al[0] = d[0] * inv;
        be[0] = -a[0] * inv;
        gm[0] = P == 1 ? -c[0] * inv : 0.f;
#pragma unroll
        for (int i = 1; i < P; ++i) {
            inv = frcp(fmaf(-a[i], cp[i - 1], b[i]));
            cp[i] = c[i] * inv;
            al[i] = fmaf(-a[i], al[i - 1], d[i]) * inv;
            be[i] = -a[i] * be[i - 1] * inv;
            gm[i] = i == P - 1 ? -c[i] * inv : 0.f;  // earlier rows have a zero right-hand side
        }
#pragma unroll
        for (int i = P - 2; i >= 0; --i) {
            al[i] = fmaf(-cp[i], al[i + 1], al[i]);
            be[i] = fmaf(-cp[i], be[i + 1], be[i]);
            gm[i] = -cp[i] * gm[i + 1];
        }
    }
    Aff Fo = Aff{al[0], be[0], gm[0]};
    Aff Lo = Aff{al[P - 1], be[P - 1], gm[P - 1]};

    // (2) merge stages: runs of S threads, RS of them per group
    const int nthr = blockDim.x;
    int par = 0;
    constexpr int LR = R >= 8 ? 3 : (R >= 4 ? 2 : 1);
#pragma unroll
    for (int log_s = 0; log_s < log_tps;) {
        const int lrs = log_tps - log_s >= LR ? LR : log_tps - log_s;  // log2 of this stage's radix
        const int rs = 1 << lrs;
        const bool by_shuffle = SHUFFLE && log_s + lrs <= 5;
        float4 *bf = buf + (2 * par) * nthr;
        float4 *bl = bf + nthr;
        if constexpr (R >= 8) {
            if (rs == 8) wm_stage<8>(Fo, Lo, t, log_s, by_shuffle, bf, bl);
        }
        if constexpr (R >= 4) {
            if (rs == 4) wm_stage<4>(Fo, Lo, t, log_s, by_shuffle, bf, bl);
        }
        if (rs == 2) wm_stage<2>(Fo, Lo, t, log_s, by_shuffle, bf, bl);
        if (!by_shuffle) par ^= 1;
        log_s += lrs;
    }

    // (3) neighbours' boundary unknowns, then the interior
    float xl_nb, xr_nb;
    if (wm_warp_only(SHUFFLE, tps)) {
        const float up = __shfl_up_sync(kFullMask, Lo.a, 1);
        const float dn = __shfl_down_sync(kFullMask, Fo.a, 1);
        xl_nb = t > 0 ? up : 0.f;
        xr_nb = t < tps - 1 ? dn : 0.f;
    } else {
        float2 *xb = reinterpret_cast<float2 *>(buf + (2 * par) * nthr);
        xb[tid] = make_float2(Fo.a, Lo.a);
        __syncthreads();
        xl_nb = t > 0 ? xb[tid - 1].y : 0.f;
        xr_nb = t < tps - 1 ? xb[tid + 1].x : 0.f;
    }
#pragma unroll
    for (int i = 0; i < P; ++i) d[i] = fmaf(gm[i], xr_nb, fmaf(be[i], xl_nb, al[i]));
}

// The same, then the unknowns stored: x points at the thread's P unknowns,
// of which the first `nval` are written (fewer than P only in the last run
// of a padded system); with `vec` false every store is element-wise (rows of
// a padded system need not be 16-byte aligned).
template <int P, int R, int SHUFFLE>
__device__ __forceinline__ void wm_solve_regs(float (&a)[P], float (&b)[P], float (&c)[P], float (&d)[P], float *x,
                                              bool active, int log_tps, float4 *buf, int nval = P,
                                              bool vec = true) {
    wm_solve_inreg<P, R, SHUFFLE>(a, b, c, d, log_tps, buf);
    if (active) {
        if (vec && nval >= P) {
            store_run<float, P>(x, d);
        } else {
#pragma unroll
            for (int i = 0; i < P; ++i)
                if (i < nval) x[i] = d[i];
        }
    }
}

// The same reading the thread's P equations from global memory (ga..gd).
template <int P, int R, int SHUFFLE>
__device__ __forceinline__ void wm_solve(const float *ga, const float *gb, const float *gc, const float *gd, float *x,
                                         bool active, int log_tps, float4 *buf) {
    float a[P], b[P], c[P], d[P];
    if (active) {
        load_run<float, P>(ga, a);
        load_run<float, P>(gb, b);
        load_run<float, P>(gc, c);
        load_run<float, P>(gd, d);
    } else {  // identity rows for unused system slots
#pragma unroll
        for (int i = 0; i < P; ++i) {
            a[i] = 0.f;
            b[i] = 1.f;
            c[i] = 0.f;
            d[i] = 0.f;
        }
    }
    wm_solve_regs<P, R, SHUFFLE>(a, b, c, d, x, active, log_tps, buf);
}

}  // namespace wm
}  // namespace bplg
