// Device building blocks of the Stockham FFT shared by the batched and the
// uneven-batch kernels: radix-2/4/8/16 DFT codelets with compile-time
// constants, the mixed-radix first stage, the Stockham output index map, and
// the padded shared-memory index.
#pragma once

#include <cuda_runtime.h>

namespace bplg {

// cos and sin of 2 pi k / 16, k = 0..4 (the other eighths follow by symmetry)
__host__ __device__ constexpr float cos16(int k) {
    switch (k & 15) {
        case 0: return 1.0f;
        case 1: return 0.92387953251128675613f;
        case 2: return 0.70710678118654752440f;
        case 3: return 0.38268343236508977173f;
        case 4: return 0.0f;
        case 5: return -0.38268343236508977173f;
        case 6: return -0.70710678118654752440f;
        case 7: return -0.92387953251128675613f;
        case 8: return -1.0f;
        case 9: return -0.92387953251128675613f;
        case 10: return -0.70710678118654752440f;
        case 11: return -0.38268343236508977173f;
        case 12: return 0.0f;
        case 13: return 0.38268343236508977173f;
        case 14: return 0.70710678118654752440f;
        default: return 0.92387953251128675613f;
    }
}
__host__ __device__ constexpr float sin16(int k) { return cos16(k - 4); }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
    return make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}

// a * exp(DIR 2 pi i k / m) for compile-time k, m in {2, 4, 8, 16}
template <int DIR, int K, int M>
__device__ __forceinline__ float2 cmul_root(float2 a) {
    constexpr int k16 = (K * (16 / M)) & 15;
    if constexpr (k16 == 0) {
        return a;
    } else if constexpr (k16 == 8) {
        return make_float2(-a.x, -a.y);
    } else if constexpr (k16 == 4) {  // w = DIR * i
        return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
    } else if constexpr (k16 == 12) {  // w = -DIR * i
        return DIR < 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
    } else {
        constexpr float c = cos16(k16);
        constexpr float s = DIR * sin16(k16);
        return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
    }
}

__host__ __device__ constexpr int bitrev(int i, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}
__host__ __device__ constexpr int clog2(int v) { return v <= 1 ? 0 : 1 + clog2(v / 2); }

// One radix-2 decimation-in-frequency layer of half-size H on R registers:
// (a, b) -> (a + b, (a - b) W_{2H}^k).
template <int R, int DIR, int H, int B0, int K>
__device__ __forceinline__ void dif_bfly(float2 (&v)[R]) {
    if constexpr (B0 < R) {
        if constexpr (K < H) {
            float2 a = v[B0 + K], b = v[B0 + K + H];
            v[B0 + K] = cadd(a, b);
            v[B0 + K + H] = cmul_root<DIR, K, 2 * H>(csub(a, b));
            dif_bfly<R, DIR, H, B0, K + 1>(v);
        } else {
            dif_bfly<R, DIR, H, B0 + 2 * H, 0>(v);
        }
    }
}
template <int R, int DIR, int H>
__device__ __forceinline__ void dif_layers(float2 (&v)[R]) {
    if constexpr (H >= 1) {
        dif_bfly<R, DIR, H, 0, 0>(v);
        dif_layers<R, DIR, H / 2>(v);
    }
}

// In-register R-point DFT, natural order in and out.
template <int R, int DIR>
__device__ __forceinline__ void dft_codelet(float2 (&v)[R]) {
    if constexpr (R > 1) {
        dif_layers<R, DIR, R / 2>(v);
        float2 t[R];
#pragma unroll
        for (int i = 0; i < R; ++i) t[i] = v[bitrev(i, clog2(R))];
#pragma unroll
        for (int i = 0; i < R; ++i) v[i] = t[i];
    }
}

// First stage with the lower radix R0 (Ns = 1, no twiddles): the thread's R
// registers hold R/R0 butterflies, butterfly q using registers q, q+Q, ...
template <int R, int R0, int DIR>
__device__ __forceinline__ void first_stage_mixed(float2 (&v)[R]) {
    constexpr int Q = R / R0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        float2 u[R0];
#pragma unroll
        for (int r = 0; r < R0; ++r) u[r] = v[q + r * Q];
        dft_codelet<R0, DIR>(u);
#pragma unroll
        for (int r = 0; r < R0; ++r) v[q + r * Q] = u[r];
    }
}

// Output position of register m after a stage.  Radix-R stage: base + m Ns.
// Mixed first stage of radix R0 = 2^lr0 (Q = R / R0 butterflies per thread):
// register m = q + r Q holds output r of butterfly j + q T, i.e. position
// (j + q T) R0 + r.
struct OutMap {
    int base, shift, mixed, lr0, lq, j, T;
    __device__ __forceinline__ int operator()(int m) const {
        if (mixed) return ((j + (m & ((1 << lq) - 1)) * T) << lr0) + (m >> lq);
        return base + (m << shift);
    }
};

template <int LAYOUT, int PAD>
__device__ __forceinline__ int pidx(int e) {
    if constexpr (!PAD) return e;
    if constexpr (LAYOUT == 0) return e + (e >> 4);
    return e + (e >> 5);
}

template <int LAYOUT, int PAD>
__host__ __device__ __forceinline__ int sig_stride(int n) {
    if (!PAD) return n;
    int p = LAYOUT == 0 ? (n >> 4) : (n >> 5);
    return n + (p > 0 ? p : 1);
}

// Compile-time stage schedule of a padded radix-R Stockham transform of
// n = 2^LOGN points (used by the size-specialised batched kernel and the
// uneven-batch kernel).  With n, the radix and every stage's stride Ns known
// at compile time, the stage loop unrolls and each exchange address is one per-thread
// padded base plus a compile-time offset.  With the padding group G (16
// float2 or 32 floats) and every stride a power of two, a stage's positions
// base + off never carry across a group boundary (base mod G + off mod G < G:
// base mod G is k < Ns plus a multiple of min(Ns R, G), off mod G at most
// G - Ns), so pad(base + off) = pad(base) + off + off / G with pad(e) =
// e + e / G; the same holds for the reads j + m T.  The generic kernel
// recomputes shifts and pads for every element, which made the large
// transforms issue-bound.
template <int R, int LOGN>
struct FftShape {
    static constexpr int LR = clog2(R);
    static constexpr int LR0 = LOGN % LR;  // radix 2^LR0 first stage when non-zero
    static constexpr int LQ = LR - LR0;
    static constexpr int LOGT = LOGN - LR;
    static constexpr int T = 1 << LOGT;
    static constexpr int NST = (LR0 ? 1 : 0) + LOGN / LR;
    static constexpr int log_ns(int st) { return st == 0 ? 0 : (LR0 ? LR0 + (st - 1) * LR : st * LR); }
};

template <int G>
__device__ __forceinline__ int pad_g(int e) {
    return e + e / G;
}

// Output positions of stage ST as (per-thread base, compile-time offset of
// register m), written to the padded exchange buffer or to global memory.
template <int R, int LOGN, int ST>
struct StageOut {
    using S = FftShape<R, LOGN>;
    static constexpr bool kMixed = ST == 0 && S::LR0 != 0;
    static constexpr int LNS = S::log_ns(ST);
    __device__ __forceinline__ static int base(int j) {
        if constexpr (kMixed) return j << S::LR0;
        else return ((j >> LNS) << (LNS + S::LR)) + (j & ((1 << LNS) - 1));
    }
    static constexpr int off(int m) {
        return kMixed ? (((m & ((1 << S::LQ) - 1)) * S::T) << S::LR0) + (m >> S::LQ) : (m << LNS);
    }
};

// The last stage hands each output, with its natural-order position, to
// store(position, value); with SYNC_LAST the block synchronises first (for a
// store into the exchange buffer that other threads may still be reading).
template <int R, int LOGN, int DIR, int LAYOUT, int ST, bool SYNC_LAST = false, class Store>
__device__ __forceinline__ void fft_fixed_stages_st(float2 (&v)[R], float2 *buf2, float *buf1, int j,
                                                    const float2 *__restrict__ tw, Store &store) {
    using S = FftShape<R, LOGN>;
    using O = StageOut<R, LOGN, ST>;
    constexpr int G = LAYOUT == 0 ? 16 : 32;
    if constexpr (O::kMixed) {
        first_stage_mixed<R, (1 << S::LR0), DIR>(v);
    } else {
        constexpr int LNS = O::LNS;
        if constexpr (LNS > 0) {
            const int k = j & ((1 << LNS) - 1);
            const float2 *twk = tw + ((1 << LNS) << S::LR);
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = __ldg(twk + r * k);
                if (DIR > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        dft_codelet<R, DIR>(v);
    }
    const int ob = O::base(j);
    if constexpr (ST == S::NST - 1) {
        if constexpr (SYNC_LAST) __syncthreads();
#pragma unroll
        for (int r = 0; r < R; ++r) store(ob + O::off(r), v[r]);
    } else {
        const int pb = pad_g<G>(ob);
        const int pj = pad_g<G>(j);
        if constexpr (LAYOUT == 0) {
            __syncthreads();
#pragma unroll
            for (int r = 0; r < R; ++r) buf2[pb + O::off(r) + O::off(r) / G] = v[r];
            __syncthreads();
#pragma unroll
            for (int m = 0; m < R; ++m) v[m] = buf2[pj + m * S::T + (m * S::T) / G];
        } else {
            __syncthreads();
#pragma unroll
            for (int r = 0; r < R; ++r) buf1[pb + O::off(r) + O::off(r) / G] = v[r].x;
            __syncthreads();
#pragma unroll
            for (int m = 0; m < R; ++m) v[m].x = buf1[pj + m * S::T + (m * S::T) / G];
            __syncthreads();
#pragma unroll
            for (int r = 0; r < R; ++r) buf1[pb + O::off(r) + O::off(r) / G] = v[r].y;
            __syncthreads();
#pragma unroll
            for (int m = 0; m < R; ++m) v[m].y = buf1[pj + m * S::T + (m * S::T) / G];
        }
        fft_fixed_stages_st<R, LOGN, DIR, LAYOUT, ST + 1, SYNC_LAST>(v, buf2, buf1, j, tw, store);
    }
}

// The stage schedule with the last stage stored straight to global memory
// (natural order, streaming stores) when `active`.
template <int R, int LOGN, int DIR, int LAYOUT, int ST>
__device__ __forceinline__ void fft_fixed_stages(float2 (&v)[R], float2 *buf2, float *buf1, int j,
                                                 const float2 *__restrict__ tw, float2 *gout, bool active) {
    auto store = [&](int pos, float2 val) {
        if (active) __stcs(gout + pos, val);
    };
    fft_fixed_stages_st<R, LOGN, DIR, LAYOUT, ST>(v, buf2, buf1, j, tw, store);
}

}  // namespace bplg
