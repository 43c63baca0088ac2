// Batched complex FFT whose radix-16 Stockham stages run on tensor cores.
//
// A radix-16 stage applies the 16-point DFT to every butterfly:
// Y[r] = sum_m X[m] W^(m r), W = exp(dir 2 pi i / 16).  In real arithmetic
// one tile of 16 butterflies is a [16 x 32] x [32 x 32] product,
//     [Yr Yi] = [Xr Xi] [[Fr, Fi], [-Fi, Fr]],  Fr = cos(2 pi m r/16),
//                                               Fi = dir sin(2 pi m r/16),
// computed with mma.sync m16n8k16 (2 k-steps x 4 n-tiles) on 16-bit inputs
// split into hi and lo parts, X = Xh + Xl, F = Fh + Fl, accumulating
// Xh Fh + Xh Fl + Xl Fh in float32 (the Xl Fl term is below the float32
// rounding of the result).  Each lane reads exactly the A-fragment elements
// it owns -- butterflies g and g+8 of its tile, inputs m = 2q, 2q+1, 2q+8,
// 2q+9 (g = lane/4, q = lane%4) -- from the Stockham exchange buffer,
// multiplies them by the float64-generated twiddles in float32, splits and
// packs them; its D fragment holds outputs r in the same set, which go back
// to the exchange buffer at the Stockham positions.  A mixed-radix first
// stage (when 4 does not divide log2 N) runs on the CUDA cores.
//
// FP16 has a small range: every tensor-core stage scales its input by 1/4
// (exact) so magnitudes stay O(1) for the growth of a 16-point DFT, and the
// output is rescaled by 4^stages at the end.  BF16 needs no scaling.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "device_util.cuh"
#include "fft_common.cuh"
#include "internal.h"
#include "tc_split.cuh"
#include "tcgen05.cuh"

namespace bplg {

template <int PREC>
struct Split;

template <>
struct Split<BPLG_TC_BF16> {
    // pack (x0, x1) -> hi pair and lo pair (lower 16 bits: x0)
    static __device__ __forceinline__ void pack(float x0, float x1, uint32_t &hi, uint32_t &lo) {
        HiLo<BPLG_TC_BF16>::pack(x0, x1, hi, lo);
    }
    static __device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
    static constexpr float kStageScale = 1.0f;
};

template <>
struct Split<BPLG_TC_F16> {
    static __device__ __forceinline__ void pack(float x0, float x1, uint32_t &hi, uint32_t &lo) {
        HiLo<BPLG_TC_F16>::pack(x0, x1, hi, lo);
    }
    static __device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
    static constexpr float kStageScale = 0.25f;
};

// Entry (m, r) of the real 32 x 32 DFT matrix for k-step ks (0: rows of Xr,
// 1: rows of Xi) and n-tile nt (0,1: columns of Yr; 2,3: columns of Yi).
template <int DIR>
__device__ __forceinline__ float dft_real_entry(int ks, int nt, int m, int r) {
    const int e = (m * r) & 15;
    const float c = cos16(e);
    const float s = DIR * sin16(e);
    if (ks == 0) return nt < 2 ? c : s;
    return nt < 2 ? -s : c;
}

// B fragments (hi and lo) of this lane for every (k-step, n-tile):
// b0 holds k = 2q, 2q+1; b1 holds k = 2q+8, 2q+9; column n = lane / 4.
template <int PREC, int DIR>
__device__ __forceinline__ void dft_b_fragments(uint32_t (&bh)[2][4][2], uint32_t (&bl)[2][4][2]) {
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, q = lane & 3;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int r = 8 * (nt & 1) + g;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m0 = 2 * q + 8 * h;
                Split<PREC>::pack(dft_real_entry<DIR>(ks, nt, m0, r), dft_real_entry<DIR>(ks, nt, m0 + 1, r),
                                  bh[ks][nt][h], bl[ks][nt][h]);
            }
        }
}

// One tensor-core radix-16 stage for the 16 butterflies b0 .. b0+15 of a
// signal (stride Ns, tile base b0): gather, twiddle, split, 24 MMAs.
// Returns this lane's outputs y[row][k] for rows g, g+8 and r in
// {2q, 2q+1, 2q+8, 2q+9} (k = 0..3 in that order).
template <int PREC, int DIR>
__device__ __forceinline__ void tc_tile(const float2 *buf, int sbase, int b0, int logNs, int logT,
                                       const float2 *__restrict__ tw, float scale, const uint32_t (&bh)[2][4][2],
                                       const uint32_t (&bl)[2][4][2], float2 (&y)[2][4]) {
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, q = lane & 3;
    const int T = 1 << logT;
    const int Ns = 1 << logNs;
    const int ms[4] = {2 * q, 2 * q + 1, 2 * q + 8, 2 * q + 9};
    float2 x[2][4];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        const int b = b0 + g + 8 * rr;
        const int k = b & (Ns - 1);
        const float2 *twp = tw + (Ns << 4);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float2 v = buf[sbase + pidx<0, 1>(b + ms[c] * T)];
            if (logNs > 0) {
                float2 w = __ldg(twp + ms[c] * k);
                if (DIR > 0) w.y = -w.y;
                v = cmul(v, w);
            }
            x[rr][c] = make_float2(v.x * scale, v.y * scale);
        }
    }
    // A fragments: ks = 0 real parts, ks = 1 imaginary parts
    uint32_t ah[2][4], al[2][4];
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const float a0 = ks ? x[rr][0].y : x[rr][0].x, a1 = ks ? x[rr][1].y : x[rr][1].x;
            const float a2 = ks ? x[rr][2].y : x[rr][2].x, a3 = ks ? x[rr][3].y : x[rr][3].x;
            Split<PREC>::pack(a0, a1, ah[ks][rr], al[ks][rr]);          // a0 / a1: cols 2q, 2q+1
            Split<PREC>::pack(a2, a3, ah[ks][2 + rr], al[ks][2 + rr]);  // a2 / a3: cols 2q+8, 2q+9
        }
    }
    float d[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
#pragma unroll
        for (int i = 0; i < 4; ++i) d[nt][i] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            const uint32_t Ah[4] = {ah[ks][0], ah[ks][1], ah[ks][2], ah[ks][3]};
            const uint32_t Al[4] = {al[ks][0], al[ks][1], al[ks][2], al[ks][3]};
            Split<PREC>::mma(d[nt], Al, bh[ks][nt][0], bh[ks][nt][1]);
            Split<PREC>::mma(d[nt], Ah, bl[ks][nt][0], bl[ks][nt][1]);
            Split<PREC>::mma(d[nt], Ah, bh[ks][nt][0], bh[ks][nt][1]);
        }
    }
    // D fragment: d[nt][0..1] row g, cols 2q, 2q+1; d[nt][2..3] row g+8.
    // nt 0 -> Yr r = 2q.., nt 1 -> Yr r = 8+2q.., nt 2/3 -> Yi likewise.
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        y[rr][0] = make_float2(d[0][2 * rr + 0], d[2][2 * rr + 0]);
        y[rr][1] = make_float2(d[0][2 * rr + 1], d[2][2 * rr + 1]);
        y[rr][2] = make_float2(d[1][2 * rr + 0], d[3][2 * rr + 0]);
        y[rr][3] = make_float2(d[1][2 * rr + 1], d[3][2 * rr + 1]);
    }
}

// Block: spb signals x T = n/16 threads (T >= 32); each warp owns two tiles
// of 16 butterflies per stage.  Input and output are staged through the
// padded exchange buffer with 16-byte global accesses.
template <int PREC, int DIR, int MAXT>
__global__ void __launch_bounds__(MAXT)
    fft_tc_kernel(const float2 *in, float2 *out, const float2 *__restrict__ tw, int logn, int spb, int64_t batch) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    const int n = 1 << logn;
    const int logT = logn - 4;
    const int T = 1 << logT;
    const int tid = threadIdx.x;
    const int s = tid >> logT;
    const int j = tid & (T - 1);
    const int64_t sig0 = static_cast<int64_t>(blockIdx.x) * spb;
    const int64_t left = batch - sig0;
    const int nvalid = left < spb ? static_cast<int>(left) : spb;
    const int stride = sig_stride<0, 1>(n);
    const int sbase = s * stride;
    const int lane = tid & 31;
    const int g = lane >> 2, q = lane & 3;
    const int wj = (j >> 5) << 5;  // first butterfly of this warp's 32 within the signal

    uint32_t bh[2][4][2], bl[2][4][2];
    dft_b_fragments<PREC, DIR>(bh, bl);

    // stage the input tile
    {
        const float4 *gsrc = reinterpret_cast<const float4 *>(in + sig0 * n);
        const int count4 = (nvalid * n) >> 1;
        for (int qq = tid; qq < count4; qq += blockDim.x) {
            const float4 w = __ldcs(gsrc + qq);
            const int e0 = qq << 1;
            const int ss = e0 >> logn;
            const int e = e0 & (n - 1);
            buf[ss * stride + pidx<0, 1>(e)] = make_float2(w.x, w.y);
            buf[ss * stride + pidx<0, 1>(e + 1)] = make_float2(w.z, w.w);
        }
    }
    __syncthreads();

    const int lr0 = logn & 3;
    int logNs = 0;
    if (lr0) {  // mixed-radix first stage on the CUDA cores (Ns = 1)
        float2 v[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = buf[sbase + pidx<0, 1>(j + m * T)];
        if (lr0 == 1) first_stage_mixed<16, 2, DIR>(v);
        if (lr0 == 2) first_stage_mixed<16, 4, DIR>(v);
        if (lr0 == 3) first_stage_mixed<16, 8, DIR>(v);
        OutMap om{0, 0, 1, lr0, 4 - lr0, j, T};
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 16; ++r) buf[sbase + pidx<0, 1>(om(r))] = v[r];
        logNs = lr0;
    }
    const int tc_stages = logn >> 2;
    const float scale = Split<PREC>::kStageScale;
    for (int st = 0; st < tc_stages; ++st) {
        __syncthreads();
        float2 y[2][2][4];
#pragma unroll
        for (int tile = 0; tile < 2; ++tile)
            tc_tile<PREC, DIR>(buf, sbase, wj + 16 * tile, logNs, logT, tw, scale, bh, bl, y[tile]);
        __syncthreads();
        const int Ns = 1 << logNs;
        const int rs[4] = {2 * q, 2 * q + 1, 2 * q + 8, 2 * q + 9};
#pragma unroll
        for (int tile = 0; tile < 2; ++tile)
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                const int b = wj + 16 * tile + g + 8 * rr;
                const int base = ((b >> logNs) << (logNs + 4)) + (b & (Ns - 1));
#pragma unroll
                for (int c = 0; c < 4; ++c) buf[sbase + pidx<0, 1>(base + (rs[c] << logNs))] = y[tile][rr][c];
            }
        logNs += 4;
    }
    __syncthreads();
    // write the tile back, undoing the per-stage scale (exact power of two)
    {
        float unscale = 1.f;
        for (int st = 0; st < tc_stages; ++st) unscale *= 1.0f / scale;
        float4 *gdst = reinterpret_cast<float4 *>(out + sig0 * n);
        const int count4 = (nvalid * n) >> 1;
        for (int qq = tid; qq < count4; qq += blockDim.x) {
            const int e0 = qq << 1;
            const int ss = e0 >> logn;
            const int e = e0 & (n - 1);
            const float2 lo = buf[ss * stride + pidx<0, 1>(e)];
            const float2 hi = buf[ss * stride + pidx<0, 1>(e + 1)];
            __stcs(gdst + qq, make_float4(lo.x * unscale, lo.y * unscale, hi.x * unscale, hi.y * unscale));
        }
    }
}

// ---------------------------------------------------------------------------
// tcgen05 variant (io 0).  One thread per butterfly, as in the float32 path:
// each thread holds its 16 inputs, multiplies them by the stage twiddles in
// float32, splits them into 16-bit hi and lo parts and writes its row of
// the A matrices [Re x_0..15 | Im x_0..15] (K = 32) to shared memory in the
// no-swizzle K-major layout.  One thread then issues, per tile of 128
// butterflies, the three split products A_lo B_hi + A_hi B_lo + A_hi B_hi
// as 2 x 3 tcgen05.mma (M = 128, N = 32, K = 16) accumulating in float32 in
// tensor memory, and commits them to an mbarrier; every thread reads its row
// of the result back with one tcgen05.ld (32 columns: Re Y_0..15, Im
// Y_0..15).  B is the real form of the 16-point DFT matrix,
//     [Re Y | Im Y] = [Re x | Im x] [[C, dir S], [-dir S, C]],
// C = cos(2 pi k n / 16), S = sin(2 pi k n / 16), also split into hi + lo.
// The A matrices reuse the exchange buffer (dead while the MMAs run); the
// exchanges between stages, the twiddles and the mixed-radix first stage are
// those of the size-specialised float32 kernel.
template <int PREC>
struct TcSplit;

template <>
struct TcSplit<BPLG_TC_BF16> {
    static constexpr uint32_t kFmt = 1;
    static constexpr float kStageScale = 1.0f;
    static __device__ __forceinline__ void pack(float x0, float x1, uint32_t &hi, uint32_t &lo) {
        Split<BPLG_TC_BF16>::pack(x0, x1, hi, lo);
    }
};

template <>
struct TcSplit<BPLG_TC_F16> {
    static constexpr uint32_t kFmt = 0;
    static constexpr float kStageScale = 0.25f;
    static __device__ __forceinline__ void pack(float x0, float x1, uint32_t &hi, uint32_t &lo) {
        Split<BPLG_TC_F16>::pack(x0, x1, hi, lo);
    }
};

// cos(2 pi e / 16), e = 0..15, as a table (the B matrix is built per block
// with data-dependent indices); sin(2 pi e / 16) = cos(2 pi (e - 4) / 16)
__device__ const float kCos16Table[16] = {cos16(0),  cos16(1),  cos16(2),  cos16(3),  cos16(4),  cos16(5),
                                          cos16(6),  cos16(7),  cos16(8),  cos16(9),  cos16(10), cos16(11),
                                          cos16(12), cos16(13), cos16(14), cos16(15)};

struct Tc5Ctx {
    unsigned char *abase;  // A hi (tiles x 8 KB), then A lo (tiles x 8 KB): aliases the exchange buffer
    unsigned char *bsm;    // B hi (2 KB), B lo (2 KB)
    uint64_t *bar;
    uint32_t tmem;
    int tiles;
    uint32_t phase;
    bool ok;
};

// The tensor-core 16-point DFT of every thread's v (in place).
template <int PREC>
__device__ __forceinline__ bool tc5_dft(float2 (&v)[16], Tc5Ctx &c) {
    const int tid = threadIdx.x;
    const int t = tid >> 7, row = tid & 127;
    __syncthreads();  // the exchange buffer's last reads are done: A may overwrite it
    {
        unsigned char *ah = c.abase + t * 8192 + umma_canon_offset(row, 0);
        unsigned char *al = ah + c.tiles * 8192;
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {  // 8 values per 16-byte chunk
            uint32_t h[4], l[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m0 = (kc & 1) * 8 + 2 * q;
                const float x0 = kc < 2 ? v[m0].x : v[m0].y;
                const float x1 = kc < 2 ? v[m0 + 1].x : v[m0 + 1].y;
                TcSplit<PREC>::pack(x0, x1, h[q], l[q]);
            }
            *reinterpret_cast<uint4 *>(ah + kc * kUmmaLbo) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4 *>(al + kc * kUmmaLbo) = make_uint4(l[0], l[1], l[2], l[3]);
        }
    }
    fence_proxy_async();  // the A rows are read by the tensor cores (async proxy)
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        tc_fence_after();
        constexpr uint32_t idesc = umma_idesc_f16(TcSplit<PREC>::kFmt, 128, 32);
        const uint32_t a0 = smem_u32(c.abase), b0 = smem_u32(c.bsm);
        for (int tt = 0; tt < c.tiles; ++tt) {
            const uint32_t d = c.tmem + static_cast<uint32_t>(tt * 32);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const uint32_t koff = ks * 2 * kUmmaLbo;
                const uint64_t ahi = umma_smem_desc(a0 + tt * 8192 + koff);
                const uint64_t alo = umma_smem_desc(a0 + c.tiles * 8192 + tt * 8192 + koff);
                const uint64_t bhi = umma_smem_desc(b0 + koff);
                const uint64_t blo = umma_smem_desc(b0 + 2048 + koff);
                umma_f16(d, alo, bhi, idesc, ks);  // the first product of a tile overwrites D
                umma_f16(d, ahi, blo, idesc, 1);
                umma_f16(d, ahi, bhi, idesc, 1);
            }
        }
        umma_commit(c.bar);
    }
    // one warp polls the mbarrier; the others wait at the barrier without
    // issuing instructions
    bool arrived = true;
    if (tid < 32) arrived = mbar_wait_bounded(c.bar, c.phase);
    const bool done = __syncthreads_and(arrived);
    if (!done) {
        c.ok = false;
        return false;
    }
    c.phase ^= 1u;
    tc_fence_after();
    uint32_t r[32];
    tmem_ld32(c.tmem + (static_cast<uint32_t>(tid & 96) << 16) + static_cast<uint32_t>(t * 32), r);
    tmem_wait_ld();
    tc_fence_before();  // ordered before the next barrier (the next stage's MMAs rewrite D)
#pragma unroll
    for (int n = 0; n < 16; ++n) v[n] = make_float2(__uint_as_float(r[n]), __uint_as_float(r[16 + n]));
    return true;
}

template <int PREC, int LOGN, int DIR, int ST>
__device__ __forceinline__ void tc5_stages(float2 (&v)[16], float2 *xbuf, int j, const float2 *__restrict__ tw,
                                           float2 *gout, bool active, Tc5Ctx &c, float unscale) {
    using S = FftShape<16, LOGN>;
    using O = StageOut<16, LOGN, ST>;
    constexpr int G = 16;
    if constexpr (O::kMixed) {
        first_stage_mixed<16, (1 << S::LR0), DIR>(v);
    } else {
        constexpr int LNS = O::LNS;
        if constexpr (LNS > 0) {
            const int k = j & ((1 << LNS) - 1);
            const float2 *twk = tw + ((1 << LNS) << 4);
#pragma unroll
            for (int r = 1; r < 16; ++r) {
                float2 w = __ldg(twk + r * k);
                if (DIR > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        if (!tc5_dft<PREC>(v, c)) return;
    }
    const int ob = O::base(j);
    if constexpr (ST == S::NST - 1) {
        if (active) {
#pragma unroll
            for (int r = 0; r < 16; ++r)
                __stcs(gout + ob + O::off(r), make_float2(v[r].x * unscale, v[r].y * unscale));
        }
    } else {
        const int pb = pad_g<G>(ob);
        const int pj = pad_g<G>(j);
        __syncthreads();  // (mixed stage) earlier readers of the buffer are done
#pragma unroll
        for (int r = 0; r < 16; ++r) xbuf[pb + O::off(r) + O::off(r) / G] = v[r];
        __syncthreads();
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = xbuf[pj + m * S::T + (m * S::T) / G];
        tc5_stages<PREC, LOGN, DIR, ST + 1>(v, xbuf, j, tw, gout, active, c, unscale);
    }
}

template <int PREC, int LOGN, int DIR, int MAXT>
__global__ void __launch_bounds__(MAXT)
    fft_tc5_kernel(const float2 *in, float2 *out, const float2 *__restrict__ tw, int logn, int spb, int64_t batch) {
    using S = FftShape<16, LOGN>;
    constexpr int N = 1 << LOGN;
    constexpr int STRIDE = N + N / 16;
    (void)logn;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x;
    const int tiles = blockDim.x >> 7;
    const uint32_t ncols = tiles <= 1 ? 32u : (tiles <= 2 ? 64u : (tiles <= 4 ? 128u : 256u));
    const int s = tid >> S::LOGT;
    const int j = tid & (S::T - 1);
    const int64_t sig = static_cast<int64_t>(blockIdx.x) * spb + s;
    const bool active = sig < batch;
    unsigned char *bsm = smem_raw;
    float2 *xall = reinterpret_cast<float2 *>(smem_raw + 4096);

    if (tid < 32) {
        tmem_alloc(&tmem_slot, ncols);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    // B = real 32 x 32 DFT matrix times the stage scale (FP16: 1/4, exact,
    // keeps the outputs' growth inside the 16-bit range), stored as rows n
    // (output column) of K = 32
    for (int e = tid; e < 32 * 32; e += blockDim.x) {
        const int n = e >> 5, k = e & 31;
        const int th = ((k & 15) * (n & 15)) & 15;
        constexpr float sc = TcSplit<PREC>::kStageScale;
        const float cs = kCos16Table[th] * sc, sn = DIR * kCos16Table[(th + 12) & 15] * sc;
        const float val = (k < 16) ? (n < 16 ? cs : sn) : (n < 16 ? -sn : cs);
        uint32_t h, l;
        TcSplit<PREC>::pack(val, 0.f, h, l);
        *reinterpret_cast<uint16_t *>(bsm + umma_canon_offset(n, k)) = static_cast<uint16_t>(h & 0xFFFFu);
        *reinterpret_cast<uint16_t *>(bsm + 2048 + umma_canon_offset(n, k)) = static_cast<uint16_t>(l & 0xFFFFu);
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    Tc5Ctx c{smem_raw + 4096, bsm, &bar, tmem_slot, tiles, 0u, true};

    float2 v[16];
    const float2 *g = in + sig * N + j;
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = active ? __ldcs(g + m * S::T) : make_float2(0.f, 0.f);
    constexpr int tc_stages = LOGN / 4;
    float unscale = 1.f;
#pragma unroll
    for (int q = 0; q < tc_stages; ++q) unscale *= 1.0f / TcSplit<PREC>::kStageScale;
    tc5_stages<PREC, LOGN, DIR, 0>(v, xall + s * STRIDE, j, tw, out + sig * N, active, c, unscale);

    tc_fence_before();
    __syncthreads();
    if (!c.ok && tid == 0) mbar_wait_bounded(&bar, c.phase);  // let a late commit land before freeing
    if (tid < 32) tmem_dealloc(c.tmem, ncols);
}

namespace {

template <int PREC, int DIR, int MAXT>
const void *tc5_func_t(int logn) {
    switch (logn) {
        case 10: return reinterpret_cast<const void *>(&fft_tc5_kernel<PREC, 10, DIR, MAXT>);
        case 11: return reinterpret_cast<const void *>(&fft_tc5_kernel<PREC, 11, DIR, MAXT>);
        case 12: return reinterpret_cast<const void *>(&fft_tc5_kernel<PREC, 12, DIR, MAXT>);
        case 13: return reinterpret_cast<const void *>(&fft_tc5_kernel<PREC, 13, DIR, MAXT>);
        case 14: return reinterpret_cast<const void *>(&fft_tc5_kernel<PREC, 14, DIR, MAXT>);
        default: return nullptr;
    }
}

template <int PREC, int DIR>
const void *tc_func_pd(int threads, int io, int logn) {
    if (io == 0) {
        if (threads % 128 != 0) return nullptr;
        return threads <= 512 ? tc5_func_t<PREC, DIR, 512>(logn) : tc5_func_t<PREC, DIR, 1024>(logn);
    }
    if (threads <= 512) return reinterpret_cast<const void *>(&fft_tc_kernel<PREC, DIR, 512>);
    return reinterpret_cast<const void *>(&fft_tc_kernel<PREC, DIR, 1024>);
}

const void *tc_func(int prec, int dir, int threads, int io, int logn) {
    if (prec == BPLG_TC_BF16)
        return dir < 0 ? tc_func_pd<BPLG_TC_BF16, -1>(threads, io, logn) : tc_func_pd<BPLG_TC_BF16, 1>(threads, io, logn);
    if (prec == BPLG_TC_F16)
        return dir < 0 ? tc_func_pd<BPLG_TC_F16, -1>(threads, io, logn) : tc_func_pd<BPLG_TC_F16, 1>(threads, io, logn);
    return nullptr;
}

}  // namespace

// the two-GEMM-pass kernels (fft_tc_gemm.cu)
const void *fft_tc_gemm_func(int prec, int dir, int logn);
int fft_tc_gemm_smem(int logn);
int fft_tc_gemm_threads(int logn);
int fft_tc_gemm_launch(const void *func, const void *in, void *out, int64_t n, int64_t batch, cudaStream_t s);

// io 1 (mma.sync): the padded exchange tile; io 0 (tcgen05): the B matrices
// (hi and lo, 4 KB) and the padded exchange tile, which the A matrices reuse;
// io 2: the 64-point DFT matrix and the data operand, both in two planes
int fft_tc_smem_bytes(int64_t n, int spb, int io) {
    if (io == 2) return fft_tc_gemm_smem(ilog2(n));
    return (io == 0 ? 4096 : 0) + spb * sig_stride<0, 1>(static_cast<int>(n)) * 8;
}

bool fft_tc_launch_info(const bplg_plan &p, int64_t n, int64_t batch, int prec, int dir, Launch *out) {
    if (!plan_structurally_valid(p, BPLG_F32, n, nullptr)) return false;
    const void *f = p.io == 2 ? fft_tc_gemm_func(prec, dir, ilog2(n)) : tc_func(prec, dir, p.L, p.io, ilog2(n));
    if (!f) return false;
    out->func = f;
    out->threads = p.io == 2 ? fft_tc_gemm_threads(ilog2(n)) : p.L;
    out->smem = fft_tc_smem_bytes(n, p.spb, p.io);
    out->blocks = (batch + p.spb - 1) / p.spb;
    return true;
}

int fft_tc_launch(const bplg_plan &p, const void *in, void *out, int64_t n, int64_t batch, int dir, int prec,
                  cudaStream_t s) {
    Launch li;
    if (!fft_tc_launch_info(p, n, batch, prec, dir, &li))
        return set_error(BPLG_ERR_INVALID_PLAN, "fft tc: plan has no kernel");
    int rc = check_grid(li.blocks, "fft tc");
    if (rc != BPLG_OK) return rc;
    if (p.io == 2) return fft_tc_gemm_launch(li.func, in, out, n, batch, s);
    const void *tw = nullptr;
    rc = twiddles_for_current_device(&tw);
    if (rc != BPLG_OK) return rc;
    rc = ensure_smem_attr(li.func, li.smem);
    if (rc != BPLG_OK) return rc;
    int logn = ilog2(n);
    int spb = p.spb;
    void *args[] = {(void *)&in, (void *)&out, (void *)&tw, &logn, &spb, &batch};
    cudaError_t e = cudaLaunchKernel(li.func, dim3(static_cast<unsigned>(li.blocks)), dim3(li.threads), args,
                                     static_cast<size_t>(li.smem), s);
    return e == cudaSuccess ? BPLG_OK : launch_error(e, "fft tc launch", li.func, li.blocks, li.threads, li.smem);
}

// Read (and optionally clear) the device error word of this file's kernels
// (the tcgen05 kernel's bounded mbarrier waits) on the current device.
int fft_tc_device_status(int *flag, bool reset) {
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
