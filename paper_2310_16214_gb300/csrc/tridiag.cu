// Batched tridiagonal solver: cyclic reduction (CR, Fig. 1(a)) down to m
// equations, parallel cyclic reduction (PCR, Fig. 1(b)) on those m, then CR
// back substitution (Section III, "Tridiagonal system solvers"; knobs of
// Section V-A).  Equation i is a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i.
//
// A block holds `spb` systems of n = 2^logn equations in shared memory as four
// arrays a, b, c, d (structure of arrays, optionally padded by one slot per 32
// against the bank conflicts of CR's doubling strides); each system is served
// by tps = n/P threads.
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
// d in place.  a_0 and c_{n-1} are never read (treated as 0).
//
// The refined variant keeps the original float32 coefficients beside a
// working copy and x in float64; each correction computes r = d - A x in
// float64, scales r by a power of two sigma so that max|r sigma| is in
// [1/2, 1), solves A e' = r sigma in float32 with the same CR/PCR code, and
// adds e = e' / sigma to x in float64.
#include "device_util.cuh"
#include "internal.h"

namespace bplg {

template <int PAD>
__device__ __forceinline__ int tpid(int i) {
    return PAD ? i + (i >> 5) : i;
}

template <int PAD>
__host__ __device__ __forceinline__ int tstride(int n) {
    if (!PAD) return n;
    int p = n >> 5;
    return n + (p > 0 ? p : 1);
}

struct SysArrays {
    float *a, *b, *c, *d;
};

// Cooperative load of the block's tile of one float array into padded rows.
template <int PAD>
__device__ __forceinline__ void tile_load(const float *g, float *sm, int arr, int arrs, int stride,
                                          int logn, int count) {
    const int n = 1 << logn;
    const int count4 = logn >= 2 ? (count >> 2) : 0;  // a float4 stays inside one row
    const float4 *g4 = reinterpret_cast<const float4 *>(g);
    for (int q = threadIdx.x; q < count4; q += blockDim.x) {
        float4 w = __ldcs(g4 + q);
        const int e = q << 2;
        const int ss = e >> logn;
        const int i = e & (n - 1);
        float *row = sm + (ss * arrs + arr) * stride;
        row[tpid<PAD>(i)] = w.x;
        row[tpid<PAD>(i + 1)] = w.y;
        row[tpid<PAD>(i + 2)] = w.z;
        row[tpid<PAD>(i + 3)] = w.w;
    }
    for (int e = (count4 << 2) + threadIdx.x; e < count; e += blockDim.x) {
        const int ss = e >> logn;
        const int i = e & (n - 1);
        sm[(ss * arrs + arr) * stride + tpid<PAD>(i)] = __ldcs(g + e);
    }
}

// CR / PCR / back substitution on the system described by `s`.  Every thread
// of the block calls this (it synchronises the block); thread t in [0, tps)
// of each system does that system's share of the work.
template <int PAD, int SHUFFLE>
__device__ void cr_pcr_solve(const SysArrays &s, int logn, int log_m, int t, int tps) {
    const int n = 1 << logn;
    const int levels = logn - log_m;
#define A_(i) s.a[tpid<PAD>(i)]
#define B_(i) s.b[tpid<PAD>(i)]
#define C_(i) s.c[tpid<PAD>(i)]
#define D_(i) s.d[tpid<PAD>(i)]
    // ---- cyclic reduction, forward
    for (int ld = 0; ld < levels; ++ld) {
        const int delta = 1 << ld;
        const int cnt = n >> (ld + 1);
        for (int u = t; u < cnt; u += tps) {
            const int i = ((u + 1) << (ld + 1)) - 1;
            const int il = i - delta;
            const int ir = i + delta;
            const float k1 = A_(i) / B_(il);
            float an = -A_(il) * k1;
            float bn = B_(i) - C_(il) * k1;
            float dn = D_(i) - D_(il) * k1;
            float cn = 0.f;
            if (ir < n) {
                const float k2 = C_(i) / B_(ir);
                bn -= A_(ir) * k2;
                dn -= D_(ir) * k2;
                cn = -C_(ir) * k2;
            }
            A_(i) = an;
            B_(i) = bn;
            C_(i) = cn;
            D_(i) = dn;
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
            const int i = ((jj + 1) << ls) - 1;
            float a = 0.f, b = 1.f, c = 0.f, d = 0.f;
            if (live) {
                a = A_(i);
                b = B_(i);
                c = C_(i);
                d = D_(i);
            }
            for (int sg = 1; sg < m; sg <<= 1) {
                const float am = __shfl_up_sync(kFullMask, a, sg, width);
                const float bm = __shfl_up_sync(kFullMask, b, sg, width);
                const float cm = __shfl_up_sync(kFullMask, c, sg, width);
                const float dm = __shfl_up_sync(kFullMask, d, sg, width);
                const float ap = __shfl_down_sync(kFullMask, a, sg, width);
                const float bp = __shfl_down_sync(kFullMask, b, sg, width);
                const float cp = __shfl_down_sync(kFullMask, c, sg, width);
                const float dp = __shfl_down_sync(kFullMask, d, sg, width);
                const bool hm = jj >= sg;
                const bool hp = jj + sg < m;
                const float k1 = hm ? a / bm : 0.f;
                const float k2 = hp ? c / bp : 0.f;
                const float an = hm ? -am * k1 : 0.f;
                const float cn = hp ? -cp * k2 : 0.f;
                const float bn = b - (hm ? cm * k1 : 0.f) - (hp ? ap * k2 : 0.f);
                const float dn = d - (hm ? dm * k1 : 0.f) - (hp ? dp * k2 : 0.f);
                a = an;
                b = bn;
                c = cn;
                d = dn;
            }
            if (live) D_(i) = d / b;
        }
        __syncthreads();
    } else {
        const int jj = t;
        const int i = ((jj + 1) << ls) - 1;
        for (int sg = 1; sg < m; sg <<= 1) {
            float an = 0.f, bn = 1.f, cn = 0.f, dn = 0.f;
            if (jj < m) {
                const float a = A_(i), b = B_(i), c = C_(i), d = D_(i);
                bn = b;
                dn = d;
                if (jj >= sg) {
                    const int im = i - (sg << ls);
                    const float k1 = a / B_(im);
                    an = -A_(im) * k1;
                    bn -= C_(im) * k1;
                    dn -= D_(im) * k1;
                }
                if (jj + sg < m) {
                    const int ip = i + (sg << ls);
                    const float k2 = c / B_(ip);
                    cn = -C_(ip) * k2;
                    bn -= A_(ip) * k2;
                    dn -= D_(ip) * k2;
                }
            }
            __syncthreads();
            if (jj < m) {
                A_(i) = an;
                B_(i) = bn;
                C_(i) = cn;
                D_(i) = dn;
            }
            __syncthreads();
        }
        if (jj < m) D_(i) = D_(i) / B_(i);
        __syncthreads();
    }
    // ---- cyclic reduction, back substitution
    for (int ld = levels - 1; ld >= 0; --ld) {
        const int delta = 1 << ld;
        const int cnt = n >> (ld + 1);
        for (int u = t; u < cnt; u += tps) {
            const int i = (u << (ld + 1)) + delta - 1;
            const float xl = (i >= delta) ? D_(i - delta) : 0.f;
            const float xr = D_(i + delta);
            D_(i) = (D_(i) - A_(i) * xl - C_(i) * xr) / B_(i);
        }
        __syncthreads();
    }
#undef A_
#undef B_
#undef C_
#undef D_
}

template <int PAD, int SHUFFLE>
__global__ void __launch_bounds__(1024)
    tridiag_kernel(const float *a, const float *b, const float *c, const float *d, float *x, int logn,
                   int log_m, int log_tps, int spb, int64_t batch) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *sm = reinterpret_cast<float *>(smem_raw);
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

    tile_load<PAD>(a + off, sm, 0, 4, stride, logn, count);
    tile_load<PAD>(b + off, sm, 1, 4, stride, logn, count);
    tile_load<PAD>(c + off, sm, 2, 4, stride, logn, count);
    tile_load<PAD>(d + off, sm, 3, 4, stride, logn, count);
    SysArrays sa;
    sa.a = sm + (s * 4 + 0) * stride;
    sa.b = sm + (s * 4 + 1) * stride;
    sa.c = sm + (s * 4 + 2) * stride;
    sa.d = sm + (s * 4 + 3) * stride;
    __syncthreads();
    if (s >= nvalid) {  // systems past the end of the batch: identity rows
        for (int i = t; i < n; i += tps) {
            sa.a[tpid<PAD>(i)] = 0.f;
            sa.b[tpid<PAD>(i)] = 1.f;
            sa.c[tpid<PAD>(i)] = 0.f;
            sa.d[tpid<PAD>(i)] = 0.f;
        }
    }
    if (t == 0) {
        sa.a[tpid<PAD>(0)] = 0.f;
        sa.c[tpid<PAD>(n - 1)] = 0.f;
    }
    __syncthreads();
    cr_pcr_solve<PAD, SHUFFLE>(sa, logn, log_m, t, tps);
    // store x (the d rows) with 16-byte accesses
    float4 *g4 = reinterpret_cast<float4 *>(x + off);
    const int count4 = logn >= 2 ? (count >> 2) : 0;
    for (int q = tid; q < count4; q += blockDim.x) {
        const int e = q << 2;
        const int ss = e >> logn;
        const int i = e & (n - 1);
        const float *row = sm + (ss * 4 + 3) * stride;
        __stcs(g4 + q, make_float4(row[tpid<PAD>(i)], row[tpid<PAD>(i + 1)], row[tpid<PAD>(i + 2)],
                                   row[tpid<PAD>(i + 3)]));
    }
    for (int e = (count4 << 2) + tid; e < count; e += blockDim.x) {
        const int ss = e >> logn;
        const int i = e & (n - 1);
        x[off + e] = sm[(ss * 4 + 3) * stride + tpid<PAD>(i)];
    }
}

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

// 2^e as float64 and float32, built from the exponent bits (exact).
__device__ __forceinline__ double pow2_f64(int e) {
    return __longlong_as_double(static_cast<long long>(1023 + e) << 52);
}
__device__ __forceinline__ float pow2_f32(int e) { return __int_as_float((127 + e) << 23); }

template <int PAD, int SHUFFLE>
__global__ void __launch_bounds__(1024)
    tridiag_refined_kernel(const float *a, const float *b, const float *c, const float *d, double *x,
                           int32_t *iters, int logn, int log_m, int log_tps, int spb, int64_t batch,
                           int max_iter, double tol) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float red[32];
    __shared__ int done_sys[32];
    float *sm = reinterpret_cast<float *>(smem_raw);
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
    // rows: [system][8][stride] floats (original a b c d, working a b c d),
    // then x as [system][n] doubles
    const int fl = spb * 8 * stride;
    double *xs_all = reinterpret_cast<double *>(sm + ((fl + 3) & ~3));
    double *xs = xs_all + s * n;

    tile_load<PAD>(a + off, sm, 0, 8, stride, logn, count);
    tile_load<PAD>(b + off, sm, 1, 8, stride, logn, count);
    tile_load<PAD>(c + off, sm, 2, 8, stride, logn, count);
    tile_load<PAD>(d + off, sm, 3, 8, stride, logn, count);
    float *oa = sm + (s * 8 + 0) * stride;
    float *ob = sm + (s * 8 + 1) * stride;
    float *oc = sm + (s * 8 + 2) * stride;
    float *od = sm + (s * 8 + 3) * stride;
    SysArrays w;
    w.a = sm + (s * 8 + 4) * stride;
    w.b = sm + (s * 8 + 5) * stride;
    w.c = sm + (s * 8 + 6) * stride;
    w.d = sm + (s * 8 + 7) * stride;
    __syncthreads();
    const bool valid = s < nvalid;
    for (int i = t; i < n; i += tps) {
        const int pi = tpid<PAD>(i);
        if (!valid) {
            oa[pi] = 0.f;
            ob[pi] = 1.f;
            oc[pi] = 0.f;
            od[pi] = 0.f;
        }
        if (i == 0) oa[pi] = 0.f;
        if (i == n - 1) oc[pi] = 0.f;
    }
    __syncthreads();
    for (int i = t; i < n; i += tps) {
        const int pi = tpid<PAD>(i);
        w.a[pi] = oa[pi];
        w.b[pi] = ob[pi];
        w.c[pi] = oc[pi];
        w.d[pi] = od[pi];
    }
    if (t == 0) done_sys[s] = valid ? 0 : 1;
    __syncthreads();
    cr_pcr_solve<PAD, SHUFFLE>(w, logn, log_m, t, tps);
    // x0 = the float32 solution; max|x0| stands for max|x| in the stopping
    // test (the corrections change x by far less than its magnitude)
    float xmaxf = 0.f;
    for (int i = t; i < n; i += tps) {
        const float v = w.d[tpid<PAD>(i)];
        xs[i] = static_cast<double>(v);
        xmaxf = fmaxf(xmaxf, fabsf(v));
    }
    xmaxf = system_max(xmaxf, red, wps);

    int applied = 0;
    for (int k = 0; k < max_iter; ++k) {
        // residual r = d - A x in float64 from the stored float32 coefficients
        float rmaxf = 0.f;
        for (int i = t; i < n; i += tps) {
            const int pi = tpid<PAD>(i);
            const double xl = i > 0 ? xs[i - 1] : 0.0;
            const double xr = i < n - 1 ? xs[i + 1] : 0.0;
            double r = static_cast<double>(od[pi]);
            r = fma(-static_cast<double>(oa[pi]), xl, r);
            r = fma(-static_cast<double>(ob[pi]), xs[i], r);
            r = fma(-static_cast<double>(oc[pi]), xr, r);
            const float rf = static_cast<float>(r);
            rmaxf = fmaxf(rmaxf, fabsf(rf));
            w.d[pi] = rf;
            w.a[pi] = oa[pi];
            w.b[pi] = ob[pi];
            w.c[pi] = oc[pi];
        }
        rmaxf = system_max(rmaxf, red, wps);
        // sigma = 2^-ex brings max|r sigma| into [1/2, 1); the exponent is
        // clamped so both powers of two stay normal
        int ex = 0;
        if (rmaxf > 0.f) frexpf(rmaxf, &ex);
        ex = ex < -120 ? -120 : (ex > 120 ? 120 : ex);
        const float sigma = pow2_f32(-ex);
        for (int i = t; i < n; i += tps) w.d[tpid<PAD>(i)] *= sigma;
        __syncthreads();
        cr_pcr_solve<PAD, SHUFFLE>(w, logn, log_m, t, tps);
        const bool was_done = done_sys[s] != 0 || rmaxf == 0.f;
        const double inv_sigma = pow2_f64(ex);
        float emaxf = 0.f;
        for (int i = t; i < n; i += tps) {
            const float ep = w.d[tpid<PAD>(i)];
            if (!was_done) xs[i] = fma(static_cast<double>(ep), inv_sigma, xs[i]);
            emaxf = fmaxf(emaxf, fabsf(ep));
        }
        emaxf = system_max(emaxf, red, wps);
        if (!was_done) ++applied;
        if (t == 0 && (was_done || static_cast<double>(emaxf) * inv_sigma <= tol * static_cast<double>(xmaxf)))
            done_sys[s] = 1;
        __syncthreads();
        int all_done = 1;
        for (int q = 0; q < spb; ++q) all_done &= done_sys[q];
        __syncthreads();
        if (all_done) break;
    }

    // store x (float64, 16-byte accesses) and the correction counts
    const int count2 = count >> 1;
    double2 *g2 = reinterpret_cast<double2 *>(x + off);
    for (int q = tid; q < count2; q += blockDim.x) {
        const int e = q << 1;
        __stcs(g2 + q, make_double2(xs_all[e], xs_all[e + 1]));
    }
    if ((count & 1) && tid == 0) x[off + count - 1] = xs_all[count - 1];
    if (iters && t == 0 && valid) iters[sig0 + s] = applied;
}

namespace {

template <int PAD>
const void *tri_func_p(int shuffle, bool refined) {
    if (refined)
        return shuffle ? reinterpret_cast<const void *>(&tridiag_refined_kernel<PAD, 1>)
                       : reinterpret_cast<const void *>(&tridiag_refined_kernel<PAD, 0>);
    return shuffle ? reinterpret_cast<const void *>(&tridiag_kernel<PAD, 1>)
                   : reinterpret_cast<const void *>(&tridiag_kernel<PAD, 0>);
}

const void *tri_func(int pad, int shuffle, bool refined) {
    if (pad < 0 || pad > 1 || shuffle < 0 || shuffle > 1) return nullptr;
    return pad ? tri_func_p<1>(shuffle, refined) : tri_func_p<0>(shuffle, refined);
}

}  // namespace

int tridiag_smem_bytes(int pad, int64_t n, int spb, bool refined) {
    const int stride = pad ? tstride<1>(static_cast<int>(n)) : static_cast<int>(n);
    if (!refined) return spb * 4 * stride * 4;
    const int fl = (spb * 8 * stride + 3) & ~3;
    return fl * 4 + spb * static_cast<int>(n) * 8;
}

bool tridiag_launch_info(const bplg_plan &p, int64_t n, int64_t batch, bool refined, Launch *out) {
    std::string why;
    bplg_plan q = p;
    if (!plan_structurally_valid(q, BPLG_F32, n, &why)) return false;
    const void *f = tri_func(p.smem_pad, p.shuffle, refined);
    if (!f) return false;
    out->func = f;
    out->threads = p.L;
    out->smem = tridiag_smem_bytes(p.smem_pad, n, p.spb, refined);
    out->blocks = (batch + p.spb - 1) / p.spb;
    return true;
}

int tridiag_launch(const bplg_plan &p, const float *a, const float *b, const float *c,
                   const float *d, float *x, int64_t n, int64_t batch, cudaStream_t s) {
    Launch li;
    if (!tridiag_launch_info(p, n, batch, false, &li))
        return set_error(BPLG_ERR_INVALID_PLAN, "tridiag: plan has no kernel");
    int rc = ensure_smem_attr(li.func, li.smem);
    if (rc != BPLG_OK) return rc;
    int logn = ilog2(n), log_m = ilog2(p.cr_switch), log_tps = ilog2(n / p.P), spb = p.spb;
    void *args[] = {(void *)&a, (void *)&b, (void *)&c, (void *)&d, (void *)&x, &logn, &log_m, &log_tps, &spb, &batch};
    cudaError_t e = cudaLaunchKernel(li.func, dim3(static_cast<unsigned>(li.blocks)), dim3(li.threads), args,
                                     static_cast<size_t>(li.smem), s);
    return e == cudaSuccess ? BPLG_OK : cuda_error(e, "tridiag launch");
}

int tridiag_refined_launch(const bplg_plan &p, const float *a, const float *b, const float *c,
                           const float *d, double *x, int64_t n, int64_t batch, int max_iter,
                           double tol, int32_t *iters, cudaStream_t s) {
    Launch li;
    if (!tridiag_launch_info(p, n, batch, true, &li))
        return set_error(BPLG_ERR_INVALID_PLAN, "tridiag refined: plan has no kernel");
    int rc = ensure_smem_attr(li.func, li.smem);
    if (rc != BPLG_OK) return rc;
    int logn = ilog2(n), log_m = ilog2(p.cr_switch), log_tps = ilog2(n / p.P), spb = p.spb;
    void *args[] = {(void *)&a,    (void *)&b,  (void *)&c,     (void *)&d,  (void *)&x,      (void *)&iters, &logn,
                    &log_m,        &log_tps,    &spb,           &batch,      &max_iter,       &tol};
    cudaError_t e = cudaLaunchKernel(li.func, dim3(static_cast<unsigned>(li.blocks)), dim3(li.threads), args,
                                     static_cast<size_t>(li.smem), s);
    return e == cudaSuccess ? BPLG_OK : cuda_error(e, "tridiag refined launch");
}

}  // namespace bplg
