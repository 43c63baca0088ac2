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
#include "tridiag_wm.cuh"

namespace bplg {

namespace {

using wm::wm_warp_only;

// RAGGED: systems of nrow < 2^logn equations (rows nrow apart), solved as
// the power-of-two system padded with identity rows (a = c = 0, b = 1,
// d = 0, whose unknowns are 0); c of the last real row is taken as 0 and
// nothing past nrow is read or written.  Accesses are 16 bytes wide when
// nrow is a multiple of 4 and P of 4, else element-wise.
template <int P, int R, int SHUFFLE, int MAXT, bool RAGGED>
__global__ void __launch_bounds__(MAXT)
    tridiag_wm_kernel(const float *ga, const float *gb, const float *gc, const float *gd, float *x, int logn,
                      int log_tps, int spb, int64_t batch, int nrow) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int s = threadIdx.x >> log_tps;
    const int t = threadIdx.x & ((1 << log_tps) - 1);
    const int64_t sig0 = static_cast<int64_t>(blockIdx.x) * spb;
    const int64_t left = batch - sig0;
    const int nvalid = left < spb ? static_cast<int>(left) : spb;
    const bool active = s < nvalid;
    float4 *buf = reinterpret_cast<float4 *>(smem_raw);
    if constexpr (!RAGGED) {
        const int64_t g0 = (sig0 + s) * (int64_t(1) << logn) + static_cast<int64_t>(t) * P;
        wm::wm_solve<P, R, SHUFFLE>(ga + g0, gb + g0, gc + g0, gd + g0, x + g0, active, log_tps, buf);
    } else {
        const int i0 = t * P;
        const int64_t g0 = (sig0 + s) * static_cast<int64_t>(nrow) + i0;
        float a[P], b[P], c[P], d[P];
        // nrow a multiple of 4: rows start on 16-byte boundaries and a group of
        // 4 equations is wholly inside or wholly past the system
        const bool vec4 = P % 4 == 0 && (nrow & 3) == 0;
        if (vec4) {
#pragma unroll
            for (int q = 0; q < (P >= 4 ? P / 4 : 0); ++q) {
                const bool in = active && i0 + 4 * q < nrow;
                float4 va = make_float4(0.f, 0.f, 0.f, 0.f), vb = make_float4(1.f, 1.f, 1.f, 1.f), vc = va, vd = va;
                if (in) {
                    va = __ldcs(reinterpret_cast<const float4 *>(ga + g0) + q);
                    vb = __ldcs(reinterpret_cast<const float4 *>(gb + g0) + q);
                    vc = __ldcs(reinterpret_cast<const float4 *>(gc + g0) + q);
                    vd = __ldcs(reinterpret_cast<const float4 *>(gd + g0) + q);
                }
                a[4 * q] = va.x; a[4 * q + 1] = va.y; a[4 * q + 2] = va.z; a[4 * q + 3] = va.w;
                b[4 * q] = vb.x; b[4 * q + 1] = vb.y; b[4 * q + 2] = vb.z; b[4 * q + 3] = vb.w;
                c[4 * q] = vc.x; c[4 * q + 1] = vc.y; c[4 * q + 2] = vc.z; c[4 * q + 3] = vc.w;
                d[4 * q] = vd.x; d[4 * q + 1] = vd.y; d[4 * q + 2] = vd.z; d[4 * q + 3] = vd.w;
            }
#pragma unroll
            for (int i = 0; i < P; ++i)
                if (i0 + i == nrow - 1) c[i] = 0.f;  // the last row's c is outside the matrix
        } else {
#pragma unroll
            for (int i = 0; i < P; ++i) {
                const bool in = active && i0 + i < nrow;
                a[i] = in ? ga[g0 + i] : 0.f;
                b[i] = in ? gb[g0 + i] : 1.f;
                c[i] = active && i0 + i < nrow - 1 ? gc[g0 + i] : 0.f;
                d[i] = in ? gd[g0 + i] : 0.f;
            }
        }
        const int nval = nrow - i0 < 0 ? 0 : (nrow - i0 < P ? nrow - i0 : P);
        wm::wm_solve_regs<P, R, SHUFFLE>(a, b, c, d, x + g0, active && nval > 0, log_tps, buf, nval, vec4);
    }
}

template <int P, int R, bool RAGGED>
const void *wm_func_r(int shuffle) {
    constexpr int MAXT = P >= 8 || R >= 8 ? 512 : 1024;
    return shuffle ? reinterpret_cast<const void *>(&tridiag_wm_kernel<P, R, 1, MAXT, RAGGED>)
                   : reinterpret_cast<const void *>(&tridiag_wm_kernel<P, R, 0, MAXT, RAGGED>);
}

template <int P, bool RAGGED>
const void *wm_func_p(int radix, int shuffle) {
    switch (radix) {
        case 2: return wm_func_r<P, 2, RAGGED>(shuffle);
        case 4: return wm_func_r<P, 4, RAGGED>(shuffle);
        case 8: return wm_func_r<P, 8, RAGGED>(shuffle);
        default: return nullptr;
    }
}

template <bool RAGGED>
const void *wm_func(int P, int radix, int shuffle) {
    switch (P) {
        case 2: return wm_func_p<2, RAGGED>(radix, shuffle);
        case 4: return wm_func_p<4, RAGGED>(radix, shuffle);
        case 8: return wm_func_p<8, RAGGED>(radix, shuffle);
        case 16: return wm_func_p<16, RAGGED>(radix, shuffle);
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
    const void *f = wm_func<false>(p.P, p.radix, p.shuffle);
    if (!f) return false;
    out->func = f;
    out->threads = p.L;
    out->smem = tridiag_wm_smem_bytes(p, n);
    out->blocks = (batch + p.spb - 1) / p.spb;
    return true;
}

int tridiag_wm_launch(const bplg_plan &p, const float *a, const float *b, const float *c, const float *d, float *x,
                      int64_t n, int64_t batch, cudaStream_t s) {
    // a plan made for the next power of two runs a length-n system padded
    const int64_t np = p.n > 0 ? p.n : n;
    if (np < n || (np != n && np / 2 >= n)) return set_error(BPLG_ERR_INVALID_PLAN, "tridiag (Wang-Mou): plan is for another n");
    Launch li;
    if (!tridiag_wm_launch_info(p, np, batch, &li))
        return set_error(BPLG_ERR_INVALID_PLAN, "tridiag (Wang-Mou): plan has no kernel");
    if (np != n) li.func = wm_func<true>(p.P, p.radix, p.shuffle);
    int rc = check_grid(li.blocks, "tridiag (Wang-Mou)");
    if (rc != BPLG_OK) return rc;
    rc = ensure_smem_attr(li.func, li.smem);
    if (rc != BPLG_OK) return rc;
    int logn = ilog2(np), log_tps = ilog2(np / p.P), spb = p.spb, nrow = static_cast<int>(n);
    void *args[] = {(void *)&a, (void *)&b, (void *)&c, (void *)&d, (void *)&x, &logn, &log_tps, &spb, &batch, &nrow};
    cudaError_t e = cudaLaunchKernel(li.func, dim3(static_cast<unsigned>(li.blocks)), dim3(li.threads), args,
                                     static_cast<size_t>(li.smem), s);
    return e == cudaSuccess ? BPLG_OK
                            : launch_error(e, "tridiag (Wang-Mou) launch", li.func, li.blocks, li.threads, li.smem);
}

}  // namespace bplg
