// Batched inclusive sum scan (Section III, "Scan Operator"; knobs of
// Section V-B).
//
// One block holds `spb` whole problems of n elements; each problem is served
// by T = n/P threads and each thread owns P consecutive elements, read and
// written with 16-byte streaming accesses.  The prefix is formed in three
// levels:
//   1. thread-serial inclusive scan of the P elements in registers;
//   2. warp-shuffle prefix of the thread totals over aligned segments of
//      min(T, 32) lanes, with the Kogge-Stone or the Ladner-Fischer circuit
//      (Fig. 1(f) / 1(d));
//   3. when T > 32, one shared-memory slot per warp (the 32-slots-per-problem
//      scheme of Section V-B) and a second shuffle prefix over the warp totals.
// int32 arithmetic wraps modulo 2^32, which is exactly the definition.
//
// Problems of any length n (not only powers of two, the identity padding of
// a non-power-of-two size): the kernel of the next power of two n' runs with
// RAGGED set; rows are n apart, elements n..n'-1 read as 0 (the identity of
// the sum) and are not written.  When n is a multiple of 4 every row starts
// on a 16-byte boundary and a 4-element group is either wholly inside the
// row or wholly past it, so the accesses stay 16 bytes wide; otherwise they
// are element-wise.
#include "device_util.cuh"
#include "internal.h"

namespace bplg {

template <typename E, int P, int PATTERN, bool RAGGED>
__global__ void __launch_bounds__(1024)
    scan_kernel(const E *in, E *out, int log_t, int spb, int64_t batch, int64_t n) {
    __shared__ E warp_tot[32];
    const int tid = threadIdx.x;
    const int tps = 1 << log_t;  // threads per problem
    const int s = tid >> log_t;
    const int t = tid & (tps - 1);
    const int64_t sig = static_cast<int64_t>(blockIdx.x) * spb + s;
    const bool active = sig < batch;
    const int64_t base = sig * n + static_cast<int64_t>(t) * P;

    E v[P];
    using V4 = typename Vec4Of<E>::type;
    const bool vec4 = RAGGED && P % 4 == 0 && (n & 3) == 0;
    if constexpr (RAGGED) {
        if (vec4) {
#pragma unroll
            for (int q = 0; q < (P >= 4 ? P / 4 : 0); ++q) {
                const bool in_row = active && t * P + 4 * q < n;
                V4 w = {};
                if (in_row) w = ld_stream(reinterpret_cast<const V4 *>(in + base) + q);
                v[4 * q] = w.x;
                v[4 * q + 1] = w.y;
                v[4 * q + 2] = w.z;
                v[4 * q + 3] = w.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < P; ++i) v[i] = (active && t * P + i < n) ? in[base + i] : E(0);
        }
    } else if (active) {
        load_run<E, P>(in + base, v);
    } else {
#pragma unroll
        for (int i = 0; i < P; ++i) v[i] = E(0);
    }
#pragma unroll
    for (int i = 1; i < P; ++i) v[i] += v[i - 1];

    const int lane = tid & 31;
    const int width = tps < 32 ? tps : 32;
    const int lane_in_seg = lane & (width - 1);
    E incl = seg_scan<PATTERN>(v[P - 1], lane_in_seg, width);
    E excl = __shfl_up_sync(kFullMask, incl, 1, width);
    if (lane_in_seg == 0) excl = E(0);

    if (tps > 32) {
        const int warp = tid >> 5;
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        const int wps = tps >> 5;
        const int wl = warp & (wps - 1);
        E w = (lane < wps) ? warp_tot[(warp - wl) + lane] : E(0);
        w = seg_scan<PATTERN>(w, lane, 32);
        E woff = __shfl_sync(kFullMask, w, wl > 0 ? wl - 1 : 0);
        if (wl == 0) woff = E(0);
        excl += woff;
    }
#pragma unroll
    for (int i = 0; i < P; ++i) v[i] += excl;
    if constexpr (RAGGED) {
        if (vec4) {
#pragma unroll
            for (int q = 0; q < (P >= 4 ? P / 4 : 0); ++q)
                if (active && t * P + 4 * q < n) {
                    V4 w;
                    w.x = v[4 * q];
                    w.y = v[4 * q + 1];
                    w.z = v[4 * q + 2];
                    w.w = v[4 * q + 3];
                    st_stream(reinterpret_cast<V4 *>(out + base) + q, w);
                }
        } else {
#pragma unroll
            for (int i = 0; i < P; ++i)
                if (active && t * P + i < n) out[base + i] = v[i];
        }
    } else if (active) {
        store_run<E, P>(out + base, v);
    }
}

namespace {

template <typename E, int P, bool RAGGED>
const void *scan_func_p(int pattern) {
    return pattern == BPLG_PATTERN_LF ? reinterpret_cast<const void *>(&scan_kernel<E, P, 1, RAGGED>)
                                      : reinterpret_cast<const void *>(&scan_kernel<E, P, 0, RAGGED>);
}

template <typename E, bool RAGGED>
const void *scan_func_t(int P, int pattern) {
    switch (P) {
        case 1: return scan_func_p<E, 1, RAGGED>(pattern);
        case 2: return scan_func_p<E, 2, RAGGED>(pattern);
        case 4: return scan_func_p<E, 4, RAGGED>(pattern);
        case 8: return scan_func_p<E, 8, RAGGED>(pattern);
        case 16: return scan_func_p<E, 16, RAGGED>(pattern);
        case 32: return scan_func_p<E, 32, RAGGED>(pattern);
        default: return nullptr;
    }
}

const void *scan_func(int dtype, int P, int pattern, bool ragged) {
    if (dtype == BPLG_I32) return ragged ? scan_func_t<int32_t, true>(P, pattern) : scan_func_t<int32_t, false>(P, pattern);
    if (dtype == BPLG_F32) return ragged ? scan_func_t<float, true>(P, pattern) : scan_func_t<float, false>(P, pattern);
    return nullptr;
}

}  // namespace

bool scan_launch_info(const bplg_plan &p, int dtype, int64_t n, int64_t batch, Launch *out) {
    std::string why;
    if (!plan_structurally_valid(p, dtype, n, &why)) return false;
    const void *f = scan_func(dtype, p.P, p.pattern, false);
    if (!f) return false;
    out->func = f;
    out->threads = p.L;
    out->smem = 0;
    out->blocks = (batch + p.spb - 1) / p.spb;
    return true;
}

int scan_launch(const bplg_plan &p, int dtype, const void *in, void *out, int64_t n, int64_t batch,
                cudaStream_t s) {
    // a plan made for the next power of two runs a length-n problem padded
    const int64_t np = p.n > 0 ? p.n : n;
    if (np < n || (np != n && np / 2 >= n)) return set_error(BPLG_ERR_INVALID_PLAN, "scan: plan is for another n");
    Launch li;
    if (!scan_launch_info(p, dtype, np, batch, &li)) return set_error(BPLG_ERR_INVALID_PLAN, "scan: plan has no kernel");
    if (np != n) li.func = scan_func(dtype, p.P, p.pattern, true);
    int rc = check_grid(li.blocks, "scan");
    if (rc != BPLG_OK) return rc;
    int log_t = ilog2(np / p.P);
    int spb = p.spb;
    void *args[] = {const_cast<void **>(&in), &out, &log_t, &spb, &batch, &n};
    cudaError_t e = cudaLaunchKernel(li.func, dim3(static_cast<unsigned>(li.blocks)), dim3(li.threads), args,
                                     0, s);
    return e == cudaSuccess ? BPLG_OK : cuda_error(e, "scan launch");
}

}  // namespace bplg
