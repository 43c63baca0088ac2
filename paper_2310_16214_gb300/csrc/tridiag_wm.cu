// Batched tridiagonal solver by divide and conquer in the manner of Wang and
// Mou (Section III lists it among BPLG's solvers, Fig. 1(e) draws its
// prefix pattern; Section V-A notes it is the solver whose radix can be
// tuned).  Equation i is a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i with
// x_{-1} = x_n = 0.
//
// A run of consecutive equations [l, h] fixes its unknowns once the two
// unknowns just outside it, X = x_{l-1} and Y = x_{h+1}, are given; by
// linearity every unknown of the run is an affine function of them,
//     x_i = alpha_i + beta_i X + gamma_i Y.
// The method starts from short runs and repeatedly merges r adjacent runs
// into one, re-expressing the unknowns in terms of the merged run's outer
// neighbours, until one run covers the system; there X = Y = 0 and
// x_i = alpha_i.
//
// Merging r runs.  Let u_k be the last unknown of run k and v_k the first
// unknown of run k+1 (k = 0 .. r-2).  Run k's descriptor gives u_k in terms
// of its own neighbours u_{k-1} (X for k = 0) and v_k, and run k+1's gives
// v_k in terms of u_k and v_{k+1} (Y for k = r-2).  A forward sweep writes
// u_k = p_k + q_k X + s_k v_k; a backward sweep from v_{r-1} = Y then gives
// every v_k and u_k as affine functions of (X, Y).  Both sweeps share the
// pivots 1 - s_k F_{k+1}.x, which stay in (0, 2) for a strictly diagonally
// dominant matrix (every |beta| + |gamma| < 1 there).
//
// GB300 mapping.  Thread t of a system owns P consecutive equations.
//  (1) It computes alpha, beta, gamma of its own run in registers with one
//      Thomas sweep for three right-hand sides (d; -a_first at the first row;
//      -c_last at the last row).
//  (2) Merge stages of radix r (the `radix` knob) combine the threads' runs.
//      Only the first and last unknown of each thread's run are carried
//      through the stages (six numbers per thread).  A stage needs from each
//      of the r runs of its group the run's first and last descriptors; they
//      come by warp shuffles while a group fits in a warp (`shuffle` knob)
//      and through shared memory otherwise (one barrier per stage, double
//      buffered).
//  (3) Once the system is one run, each thread's first and last unknowns
//      are known; the interior ones follow from the thread's own alpha,
//      beta, gamma and its neighbours' boundary values.  The method's
//      stage-by-stage re-expression of the interior unknowns is applied once
//      at the end instead, which gives the same values in exact arithmetic.
// Divisions use the hardware reciprocal (about 1 ulp), as in the CR solver.
#include <string>

#include "device_util.cuh"
#include "internal.h"
#include "tridiag_common.cuh"

namespace bplg {

namespace {

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

template <int P, int R, int SHUFFLE, int MAXT>
__global__ void __launch_bounds__(MAXT)
    tridiag_wm_kernel(const float *ga, const float *gb, const float *gc, const float *gd, float *x, int logn,
                      int log_tps, int spb, int64_t batch) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = 1 << logn;
    const int tps = 1 << log_tps;
    const int tid = threadIdx.x;
    const int s = tid >> log_tps;
    const int t = tid & (tps - 1);
    const int64_t sig0 = static_cast<int64_t>(blockIdx.x) * spb;
    const int64_t left = batch - sig0;
    const int nvalid = left < spb ? static_cast<int>(left) : spb;
    const bool active = s < nvalid;
    const int64_t g0 = (sig0 + s) * n + static_cast<int64_t>(t) * P;

    float a[P], b[P], c[P], d[P];
    if (active) {
        load_run<float, P>(ga + g0, a);
        load_run<float, P>(gb + g0, b);
        load_run<float, P>(gc + g0, c);
        load_run<float, P>(gd + g0, d);
    } else {  // identity rows for the block's unused system slots
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
    float4 *buf = reinterpret_cast<float4 *>(smem_raw);
    const int nthr = blockDim.x;
    int par = 0;
    constexpr int LR = R >= 8 ? 3 : (R >= 4 ? 2 : 1);
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
    float xv[P];
#pragma unroll
    for (int i = 0; i < P; ++i) xv[i] = fmaf(gm[i], xr_nb, fmaf(be[i], xl_nb, al[i]));
    if (active) store_run<float, P>(x + g0, xv);
}

template <int P, int R>
const void *wm_func_r(int shuffle) {
    constexpr int MAXT = P >= 8 || R >= 8 ? 512 : 1024;
    return shuffle ? reinterpret_cast<const void *>(&tridiag_wm_kernel<P, R, 1, MAXT>)
                   : reinterpret_cast<const void *>(&tridiag_wm_kernel<P, R, 0, MAXT>);
}

template <int P>
const void *wm_func_p(int radix, int shuffle) {
    switch (radix) {
        case 2: return wm_func_r<P, 2>(shuffle);
        case 4: return wm_func_r<P, 4>(shuffle);
        case 8: return wm_func_r<P, 8>(shuffle);
        default: return nullptr;
    }
}

const void *wm_func(int P, int radix, int shuffle) {
    switch (P) {
        case 2: return wm_func_p<2>(radix, shuffle);
        case 4: return wm_func_p<4>(radix, shuffle);
        case 8: return wm_func_p<8>(radix, shuffle);
        case 16: return wm_func_p<16>(radix, shuffle);
        default: return nullptr;
    }
}

}  // namespace

int tridiag_wm_smem_bytes(const bplg_plan &p, int64_t n) {
    const int64_t tps = n / p.P;
    return wm_warp_only(p.shuffle, tps) ? 0 : 4 * 16 * p.L;
}

bool tridiag_wm_launch_info(const bplg_plan &p, int64_t n, int64_t batch, Launch *out) {
    if (!plan_structurally_valid(p, BPLG_F32, n, nullptr)) return false;
    const void *f = wm_func(p.P, p.radix, p.shuffle);
    if (!f) return false;
    out->func = f;
    out->threads = p.L;
    out->smem = tridiag_wm_smem_bytes(p, n);
    out->blocks = (batch + p.spb - 1) / p.spb;
    return true;
}

int tridiag_wm_launch(const bplg_plan &p, const float *a, const float *b, const float *c, const float *d, float *x,
                      int64_t n, int64_t batch, cudaStream_t s) {
    Launch li;
    if (!tridiag_wm_launch_info(p, n, batch, &li))
        return set_error(BPLG_ERR_INVALID_PLAN, "tridiag (Wang-Mou): plan has no kernel");
    int rc = ensure_smem_attr(li.func, li.smem);
    if (rc != BPLG_OK) return rc;
    int logn = ilog2(n), log_tps = ilog2(n / p.P), spb = p.spb;
    void *args[] = {(void *)&a, (void *)&b, (void *)&c, (void *)&d, (void *)&x, &logn, &log_tps, &spb, &batch};
    cudaError_t e = cudaLaunchKernel(li.func, dim3(static_cast<unsigned>(li.blocks)), dim3(li.threads), args,
                                     static_cast<size_t>(li.smem), s);
    return e == cudaSuccess ? BPLG_OK
                            : launch_error(e, "tridiag (Wang-Mou) launch", li.func, li.blocks, li.threads, li.smem);
}

}  // namespace bplg
