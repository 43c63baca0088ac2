// Tensor-core FFT of 4096 and 16384 points as two passes of 64-point DFTs,
// each pass one chain of tcgen05 matrix products (plan io 2 of the
// tensor-core FFT).
//
// A 4096-point transform is the 64 x 64 factorisation (the four-step form
// of the Stockham algorithm with radix 64): with n = n1 + 64 n2 and
// k = k2 + 64 k1,
//     Y[n1][k2] = sum_n2 x[n1 + 64 n2] W64^(n2 k2)            (pass 1)
//     X[k2 + 64 k1] = sum_n1 W4096^(n1 k2) Y[n1][k2] W64^(n1 k1)   (pass 2)
// with W_m = exp(dir 2 pi i / m).  A 16384-point transform first runs a
// radix-4 stage on the CUDA cores (y_m[k] = W16384^(m k) sum_q x[k + 4096 q]
// W4^(q m)), then the four 4096-point transforms of y_0 .. y_3, whose
// output k' is X[4 k' + m].
//
// Each 64-point DFT is a real product with the 128 x 128 matrix F whose row
// 2k (2k + 1) gives the real (imaginary) part of output k from the inputs'
// real parts (K columns 0..63) and imaginary parts (64..127).  Operands are
// split into 16-bit hi and lo parts (tc_split.cuh) and every product is
// Fl Dh + Fh Dl + Fh Dh, accumulated in float32 in tensor memory.  F sits in
// tensor memory (the A operand, one row per lane); the data are the B
// operand in shared memory (K-major, 16-byte core matrices without
// swizzle), so the tensor cores read one operand from shared memory:
//   pass 1: D1 = F B1^T, B1 row (sub-signal, n1), K = [re n2 | im n2];
//           D1 row (k2, part), column (sub-signal, n1)
//   pass 2: D2 = F A2^T, A2 row (sub-signal, k2) = the twiddled pass-1
//           output, K = [re n1 | im n1]; D2 row (k1, part), column
//           (sub-signal, k2)
// Between the passes each thread reads one row of D1 from tensor memory,
// swaps halves with its neighbour lane (rows 2k and 2k + 1 hold the real
// and imaginary parts), applies the twiddles in float32 (from the
// float64-generated table, kept in shared memory), splits and writes its row
// of A2 into the same buffer.  After pass 2 the same swap leaves each pair
// of lanes sixteen consecutive outputs.
//
// Blocks are persistent (one per SM, 512 worker threads) and load the next
// tile -- two 4096-point signals or one 16384-point signal -- into
// registers while the tensor cores run the current one.  The workers fill a
// buffer and arrive on an mbarrier; one thread waits on it, issues the
// products and commits them to a second mbarrier, on which the workers wait.
//   4096 points: a 17th warp issues.  Two tiles are in flight, with two data
//     buffers and two tensor-memory slots: tile i + 1 is prepared and its
//     pass 1 runs while tile i's pass 2 runs and is written out, through the
//     freed buffer, in whole lines.
//   16384 points: one lane of worker warp 0 issues (a 17th warp would cap
//     the registers at 96, too few for the prefetched tile).  A tile runs in
//     halves (quarters 0-1 and 2-3 of the radix-4 output), each pass as two
//     products of N = 128, so the CUDA cores work on one half while the
//     tensor cores run the other; the halves of D rotate through three
//     128-column blocks of tensor memory, so that the next tile's first
//     product runs while this tile's output is read and written.
// Waits on the barriers are bounded: on a timeout the block records the
// device error word and runs on without waiting, through the same barriers.
#include "device_util.cuh"
#include "fft_common.cuh"
#include "internal.h"
#include "tc_split.cuh"
#include "tcgen05.cuh"

namespace bplg {

namespace {

constexpr int kGemmThreads = 512;  // worker threads (16 warps)
constexpr int kGemmK = 128;                     // real K of a 64-point DFT
constexpr uint32_t kGemmSbo = 2048;             // bytes between 8-row groups (K = 128)

// byte offset of element (row, k) of a K-major operand with K = 128
__host__ __device__ constexpr uint32_t gemm_off(int row, int k) {
    return static_cast<uint32_t>((row >> 3) * kGemmSbo + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// shared-memory descriptor of such an operand: LBO 128 bytes (next core
// matrix along K), SBO 2048 bytes (next 8 rows), no swizzle
__device__ __forceinline__ uint64_t gemm_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((addr >> 4) & 0x3FFFu);
    d |= static_cast<uint64_t>((128u >> 4) & 0x3FFFu) << 16;
    d |= static_cast<uint64_t>((kGemmSbo >> 4) & 0x3FFFu) << 32;
    d |= static_cast<uint64_t>(1) << 46;
    return d;
}

template <int LOGN>
struct GemmShape {
    static constexpr int SIG = LOGN == 12 ? 2 : 1;       // signals per tile
    static constexpr int ROWS = LOGN == 12 ? 128 : 256;  // pass-1 columns = pass-2 rows of a tile
    static constexpr int NBUF = LOGN == 12 ? 2 : 1;      // tiles in flight (data buffers, tensor-memory slots)
    static constexpr int PLANE = ROWS * kGemmK * 2;      // one 16-bit plane of a tile's data operand
    static constexpr int SLOT_COLS = ROWS;               // tensor-memory columns of one tile's D
    // 4096 points: a 17th warp issues the products (96 registers a thread);
    // 16384 points: one lane of warp 0 does, leaving 128 registers a thread
    // for the prefetched tile
    static constexpr bool ISSUER_WARP = LOGN == 12;
    static constexpr int BLOCK = kGemmThreads + (ISSUER_WARP ? 32 : 0);
};

// tensor memory: F at columns 0..127 (hi planes 0..63, lo 64..127, two
// 16-bit K elements per column), then NBUF slots of D (4096 points), or
// three blocks of 128 columns that the halves of D rotate through (16384
// points)
constexpr uint32_t kGemmTmemCols = 512;
constexpr uint32_t kGemmFCols = 128;

// shared memory: the twiddles W4096^(n1 k2) between the passes (64 rows of
// 65, the pad keeping rows 8 apart on other banks), then NBUF data buffers
// of two planes each.  16384 points add the 3 x 64 tables W16384^(m n1) and
// W256^(m n2), m = 1..3, whose product is the radix-4 twiddle W16384^(m k),
// k = n1 + 64 n2.  (Shared memory is kept well below the maximum: what is
// left is the L1 cache, and the loads of the next tile, up to 128 KB in
// flight per SM, need it.)
constexpr int kTwStride = 65;
constexpr int kTwBytes = 64 * kTwStride * 8;
constexpr int kTw14Bytes = 2 * 3 * 64 * 8;
template <int LOGN>
constexpr int gemm_smem_bytes() {
    return kTwBytes + GemmShape<LOGN>::NBUF * 2 * GemmShape<LOGN>::PLANE + (LOGN == 14 ? kTw14Bytes : 0);
}

// eight values (one K chunk) split and stored to both planes
template <int PREC>
__device__ __forceinline__ void put_chunk(unsigned char *hi_plane, unsigned char *lo_plane, uint32_t off,
                                          const float (&x)[8]) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) HiLo<PREC>::pack(x[2 * q], x[2 * q + 1], h[q], l[q]);
    *reinterpret_cast<uint4 *>(hi_plane + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(lo_plane + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr)
                 : "memory");
}

// W_m^e = exp(DIR 2 pi i e / m) from the table of exp(-2 pi i e / m)
template <int DIR>
__device__ __forceinline__ float2 root(const float2 *__restrict__ tw, int m, int e) {
    float2 w = __ldg(tw + m + e);
    if (DIR > 0) w.y = -w.y;
    return w;
}

// issue the products of one pass on the calling thread: D = F B^T over
// K = 128 with F in tensor memory, 8 steps of K = 16 (8 tensor-memory
// columns of F, 256 bytes of B per step), three split products each
__device__ __forceinline__ void gemm_pass(uint32_t d, uint32_t f_tmem, uint64_t b_hi, uint64_t b_lo,
                                          uint32_t idesc) {
#pragma unroll
    for (int ks = 0; ks < kGemmK / 16; ++ks) {
        const uint32_t a_hi = f_tmem + static_cast<uint32_t>(8 * ks), a_lo = a_hi + 64;
        const uint64_t k = static_cast<uint64_t>(ks) * (256 >> 4);
        umma_f16_ts(d, a_lo, b_hi + k, idesc, ks > 0 ? 1u : 0u);
        umma_f16_ts(d, a_hi, b_lo + k, idesc, 1u);
        umma_f16_ts(d, a_hi, b_hi + k, idesc, 1u);
    }
}

// barrier of the worker warps alone (named barrier 1)
__device__ __forceinline__ void workers_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kGemmThreads) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// wait for the completion of phase `phase` of `bar` (bounded; one lane of
// the warp polls), then flip it.  After a timeout (ok false) nothing is
// waited for any more: the warp runs on through the same barriers as the
// others and the block ends with the device error word set.
__device__ __forceinline__ void gemm_wait(uint64_t *bar, uint32_t &phase, bool &ok) {
    if (ok) {
        bool got = true;
        if ((threadIdx.x & 31) == 0) got = mbar_wait_bounded(bar, phase);
        ok = __shfl_sync(kFullMask, got ? 1 : 0, 0) != 0;
    }
    phase ^= 1u;
}

template <int PREC, int DIR, int LOGN>
__global__ void __launch_bounds__(GemmShape<LOGN>::BLOCK, 1)
    fft_tc_gemm_kernel(const float2 *__restrict__ in, float2 *__restrict__ out, const float2 *__restrict__ tw,
                       int64_t batch) {
    using G = GemmShape<LOGN>;
    constexpr int N = 1 << LOGN;
    extern __shared__ __align__(128) unsigned char smem[];
    float2 *tws = reinterpret_cast<float2 *>(smem);  // [n1][k2], rows kTwStride apart
    unsigned char *dbuf = smem + kTwBytes;           // buffer b: hi plane, lo plane
    // 16384 points: W16384^(m n1) at [m - 1][n1], W256^(m n2) at [3 + m - 1][n2]
    float2 *tw14 = reinterpret_cast<float2 *>(dbuf + G::NBUF * 2 * G::PLANE);  // 16384 points
    // ready[b]: the workers have filled buffer b (and are done reading slot
    // b); done[b]: the products over buffer b have completed
    __shared__ __align__(8) uint64_t ready[2];
    __shared__ __align__(8) uint64_t done[2];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t ntiles = (batch + G::SIG - 1) / G::SIG;

    if (warp == 0) {
        tmem_alloc(&tmem_slot, kGemmTmemCols);
        tmem_relinquish();
    }
    if (tid == 0) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            mbar_init(&ready[b], kGemmThreads / 32);  // one arrival per worker warp
            mbar_init(&done[b], 1);
        }
        fence_mbar_init();
    }
    for (int e = tid; e < 64 * 64; e += G::BLOCK)
        tws[(e >> 6) * kTwStride + (e & 63)] = root<DIR>(tw, 4096, (e >> 6) * (e & 63));
    if constexpr (LOGN == 14) {
        for (int e = tid; e < 3 * 64; e += G::BLOCK) {
            const int m = e / 64 + 1, j = e % 64;
            tw14[e] = root<DIR>(tw, 16384, m * j);
            tw14[3 * 64 + e] = root<DIR>(tw, 256, m * j);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t tq = static_cast<uint32_t>(32 * (warp & 3)) << 16;  // this warp's tensor-memory lanes
    // F into tensor memory: row r = 2k + part_out in lane r, K column c =
    // 64 part_in + n (W = exp(DIR 2 pi i k n / 64)) in column c / 2 of the hi
    // or the lo half; each worker warp writes 32 columns of its lane quarter
    if (warp < kGemmThreads / 32) {
        const int r = 32 * (warp & 3) + lane;
        const int col0 = 32 * (warp >> 2);  // of the 128 F columns
        uint32_t w32[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int col = col0 + j, c = 2 * (col & 63);
            float f[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = r >> 1, po = r & 1, pi = (c + h) >> 6, n = (c + h) & 63;
                const float2 w = root<DIR>(tw, 64, (k * n) & 63);
                f[h] = po == 0 ? (pi == 0 ? w.x : -w.y) : (pi == 0 ? w.y : w.x);
            }
            uint32_t hi, lo;
            HiLo<PREC>::pack(f[0], f[1], hi, lo);
            w32[j] = col < 64 ? hi : lo;
        }
        tmem_st32(tmem + tq + static_cast<uint32_t>(col0), w32);
        tmem_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    uint32_t ph_ready[2], ph_done[2];
#pragma unroll
    for (int b = 0; b < 2; ++b) ph_ready[b] = ph_done[b] = 0u;
    bool ok = true;

    auto plane_hi = [&](int b) { return dbuf + b * 2 * G::PLANE; };
    auto plane_lo = [&](int b) { return dbuf + b * 2 * G::PLANE + G::PLANE; };

    // ---- loads: LOGN 12: signal u, n1 pair (2np, 2np+1), n2 = 8g .. 8g+7 as
    // 16-byte loads; LOGN 14: n1, n2 = 8g .. 8g+7, all four quarters
    constexpr int NV = LOGN == 12 ? 8 : 16;
    float4 v[NV];
    auto load = [&](int64_t tile) {
        if constexpr (LOGN == 12) {
            const int u = tid >> 8, g = (tid >> 5) & 7, np = tid & 31;
            const int64_t sig = tile * 2 + u;
            const float4 *src = reinterpret_cast<const float4 *>(in + sig * N + 2 * np + 64 * 8 * g);
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = sig < batch ? __ldcs(src + 32 * i) : make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            const int g = tid >> 6, n1 = tid & 63;
            const float2 *src = in + tile * N + n1 + 64 * 8 * g;
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int q = 0; q < 4; q += 2) {
                    const float2 a = __ldcs(src + 64 * i + 4096 * q), b = __ldcs(src + 64 * i + 4096 * (q + 1));
                    v[2 * i + q / 2] = make_float4(a.x, a.y, b.x, b.y);
                }
        }
    };

    // ---- 16384 points: the radix-4 first stage in place (v[2i] <- y0, y1
    // and v[2i + 1] <- y2, y3 of n2 = 8g + i, g = tid / 64, n1 = tid % 64)
    auto radix4 = [&]() {
        const int g = tid >> 6, n1 = tid & 63;
        const float2 w1 = tw14[n1], w2 = tw14[64 + n1], w3 = tw14[128 + n1];  // W16384^(m n1)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float4 p01 = v[2 * i], p23 = v[2 * i + 1];
            const float2 a0 = make_float2(p01.x, p01.y), a1 = make_float2(p01.z, p01.w);
            const float2 a2 = make_float2(p23.x, p23.y), a3 = make_float2(p23.z, p23.w);
            const float2 s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = csub(a1, a3);
            // DIR i (a1 - a3)
            const float2 jd = DIR < 0 ? make_float2(d13.y, -d13.x) : make_float2(-d13.y, d13.x);
            const int n2 = 8 * g + i;  // W256^(m n2)
            const float2 y0 = cadd(s02, s13);
            const float2 y1 = cmul(cadd(d02, jd), cmul(w1, tw14[3 * 64 + n2]));
            const float2 y2 = cmul(csub(s02, s13), cmul(w2, tw14[4 * 64 + n2]));
            const float2 y3 = cmul(csub(d02, jd), cmul(w3, tw14[5 * 64 + n2]));
            v[2 * i] = make_float4(y0.x, y0.y, y1.x, y1.y);
            v[2 * i + 1] = make_float4(y2.x, y2.y, y3.x, y3.y);
        }
    };
    // pass-1 operand rows m * 64 + n1 of quarters m = m0, m0 + 1: the
    // thread's eight consecutive n2 form one 16-byte chunk per plane and part
    auto put_quarters = [&](int b, int m0) {
        unsigned char *hp = plane_hi(b), *lp = plane_lo(b);
        const int g = tid >> 6, n1 = tid & 63;
#pragma unroll
        for (int m = m0; m < m0 + 2; ++m) {
            float re[8], im[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float4 q = v[2 * i + (m >> 1)];
                re[i] = (m & 1) ? q.z : q.x;
                im[i] = (m & 1) ? q.w : q.y;
            }
            put_chunk<PREC>(hp, lp, gemm_off(m * 64 + n1, 8 * g), re);
            put_chunk<PREC>(hp, lp, gemm_off(m * 64 + n1, 64 + 8 * g), im);
        }
    };

    // ---- pass-1 operand of the loaded tile: row (sub-signal, n1), K = [re n2 | im n2]
    auto prep = [&](int b) {
        unsigned char *hp = plane_hi(b), *lp = plane_lo(b);
        if constexpr (LOGN == 12) {
            const int u = tid >> 8, g = (tid >> 5) & 7, np = tid & 31;
            // the thread's rows 2np and 2np + 1, the odd one first in every
            // other group of four lanes: a warp's stores then cover all eight
            // 16-byte bank slots
            const int first = (np >> 2) & 1;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int odd = h ^ first;
                const int row = u * 64 + 2 * np + odd;
                float re[8], im[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    re[i] = odd ? v[i].z : v[i].x;
                    im[i] = odd ? v[i].w : v[i].y;
                }
                put_chunk<PREC>(hp, lp, gemm_off(row, 8 * g), re);
                put_chunk<PREC>(hp, lp, gemm_off(row, 64 + 8 * g), im);
            }
        } else {
            radix4();
            put_quarters(b, 0);
            put_quarters(b, 2);
        }
    };

    // ---- one pass over buffer b into slot b: D = F x B^T, N = ROWS (pass 1
    // with the data, pass 2 with the twiddled pass-1 output in the buffer)
    auto issue = [&](int b, uint64_t bh, uint64_t bl) {
        gemm_pass(tmem + kGemmFCols + static_cast<uint32_t>(b * G::SLOT_COLS), tmem, bh, bl,
                  umma_idesc_f16(HiLo<PREC>::kFmt, 128, G::ROWS));
        umma_commit(&done[b]);
    };
    // 16384 points: half hf of a pass, operand rows 128 hf .. 128 hf + 127,
    // into tensor-memory block blk, committed to done[hf]
    auto issue_half = [&](int hf, int blk) {
        const uint64_t off = static_cast<uint64_t>(hf) * (gemm_off(128, 0) >> 4);
        gemm_pass(tmem + kGemmFCols + static_cast<uint32_t>(128 * blk), tmem,
                  gemm_desc(smem_u32(plane_hi(0))) + off, gemm_desc(smem_u32(plane_lo(0))) + off,
                  umma_idesc_f16(HiLo<PREC>::kFmt, 128, 128));
        umma_commit(&done[hf]);
    };

    // ---- D1 row (k2, part), columns (sub-signal, n1) -> twiddled A2 rows in buffer b
    // (16384 points: half hf, quarters 2 hf and 2 hf + 1, in block blk)
    auto epi1 = [&](int b, int hf = 0, int blk = 0) {
        unsigned char *hp = plane_hi(b), *lp = plane_lo(b);
        const int r = 32 * (warp & 3) + lane;  // D1 row of this thread
        const int k2 = r >> 1, odd = r & 1;
        constexpr int CPW = 32;  // columns per warp: each lane quarter is read by 4 warps
        const int c0 = CPW * (warp >> 2);
        const uint32_t cbase = LOGN == 12 ? static_cast<uint32_t>(b * G::SLOT_COLS) : static_cast<uint32_t>(128 * blk);
#pragma unroll
        for (int h = 0; h < CPW / 16; ++h) {
            const int cb = c0 + 16 * h;  // 16 columns of one sub-signal
            uint32_t raw[16];
            tmem_ld16(tmem + tq + kGemmFCols + cbase + static_cast<uint32_t>(cb), raw);
            tmem_wait_ld();
            const int u = 2 * hf + (cb >> 6);
            const int nb = (cb & 63) + 8 * odd;  // this thread keeps n1 = nb .. nb + 7
            float re[8], im[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const uint32_t send = odd ? raw[t] : raw[8 + t];
                const float got = __uint_as_float(__shfl_xor_sync(kFullMask, send, 1));
                const float2 z = odd ? make_float2(got, __uint_as_float(raw[8 + t]))
                                     : make_float2(__uint_as_float(raw[t]), got);
                const float2 zt = cmul(z, tws[(nb + t) * kTwStride + k2]);
                re[t] = zt.x;
                im[t] = zt.y;
            }
            const int row = u * 64 + k2;  // pass-2 operand row (sub-signal, k2)
            put_chunk<PREC>(hp, lp, gemm_off(row, nb), re);
            put_chunk<PREC>(hp, lp, gemm_off(row, 64 + nb), im);
        }
    };

    // ---- D2 row (k1, part), columns = pass-2 operand rows -> X of `tile`.
    // 4096 points: staged in buffer b (free once pass 2 has completed) in
    // output order, then copied out in whole lines; staging row (sub-signal,
    // k1) of 64 outputs, its 16-byte units XOR-swizzled by (row % 4) * 2 so
    // that the lanes of a quarter warp (four rows, two units each) hit eight
    // different bank groups.  16384 points: written directly.
    constexpr int ROWB = 512;                      // bytes per staging row
    constexpr int UNITS = 2 * G::PLANE / 16;       // 16-byte units of a tile's output
    auto stage_at = [&](int b, int row, int unit) {
        return plane_hi(b) + row * ROWB + 16 * (unit ^ ((row & 3) << 1));  // both planes, contiguous
    };
    // (16384 points: quarters 0-1 in block blk_a, 2-3 in blk_b)
    auto epi2 = [&](int b, int64_t tile, int blk_a = 0, int blk_b = 0) {
        const int r = 32 * (warp & 3) + lane;
        const int k1 = r >> 1, odd = r & 1;
        constexpr int CPW = G::ROWS / 4;
        const int c0 = CPW * (warp >> 2);
#pragma unroll
        for (int h = 0; h < CPW / 16; ++h) {
            const int cb = c0 + 16 * h;
            // x[p], p = 0..15: sixteen consecutive outputs of this lane's part
            // (4096 points: columns cb + p; 16384 points: X[4 (kb + j) + u] =
            // column 64 u + kb + j, p = 4 j + u, kb = cb / 4)
            uint32_t raw[16];
            if constexpr (LOGN == 12) {
                tmem_ld16(tmem + tq + kGemmFCols + static_cast<uint32_t>(b * G::SLOT_COLS + cb), raw);
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    tmem_ld4(tmem + tq + kGemmFCols +
                                 static_cast<uint32_t>(128 * (u < 2 ? blk_a : blk_b) + 64 * (u & 1) + cb / 4),
                             &raw[4 * u]);
            }
            tmem_wait_ld();
            auto x = [&](int p) { return LOGN == 12 ? raw[p] : raw[4 * (p & 3) + (p >> 2)]; };
            // the even lane keeps outputs p = 4t + {0, 1}, the odd lane
            // 4t + {2, 3} (t = 0..3)
            float2 z[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int mine = 4 * (t >> 1) + (t & 1);  // even lane's output; + 2 for the odd lane
                const uint32_t send = odd ? x(mine) : x(mine + 2);
                const float got = __uint_as_float(__shfl_xor_sync(kFullMask, send, 1));
                z[t] = odd ? make_float2(got, __uint_as_float(x(mine + 2))) : make_float2(__uint_as_float(x(mine)), got);
            }
            if constexpr (LOGN == 14) {
                // written directly (the buffer already holds the next tile's
                // quarters 0-1): each pair of lanes fills one 32-byte sector
                // per store
                float2 *dst = out + tile * N + 256 * k1 + cb + 2 * odd;
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    __stcs(reinterpret_cast<float4 *>(dst + 4 * t),
                           make_float4(z[2 * t].x, z[2 * t].y, z[2 * t + 1].x, z[2 * t + 1].y));
                continue;
            }
            const int row = (cb >> 6) * 64 + k1;  // (sub-signal, k1)
            const int unit0 = (cb & 63) >> 1;
#pragma unroll
            for (int t = 0; t < 4; ++t)
                *reinterpret_cast<float4 *>(stage_at(b, row, unit0 + 2 * t + odd)) =
                    make_float4(z[2 * t].x, z[2 * t].y, z[2 * t + 1].x, z[2 * t + 1].y);
        }
        if constexpr (LOGN == 14) return;
        workers_sync();
        float4 *dst = reinterpret_cast<float4 *>(out + tile * (G::SIG * N));
        constexpr int UPR = ROWB / 16;  // units per row
#pragma unroll
        for (int j0 = 0; j0 < UNITS / kGemmThreads; j0 += 4) {
            float4 w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int u = tid + kGemmThreads * (j0 + j);
                w[j] = *reinterpret_cast<const float4 *>(stage_at(b, u / UPR, u % UPR));
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int u = tid + kGemmThreads * (j0 + j);
                const bool live = LOGN == 12 ? tile * 2 + u / (UNITS / 2) < batch : true;
                if (live) __stcs(dst + u, w[j]);
            }
        }
        workers_sync();  // the buffer may be refilled
    };

    // ---- the pipeline.  The workers fill a buffer (or finish reading a
    // slot) and arrive on its `ready` barrier after a proxy fence and a
    // tensor-memory fence; the issuing warp (the 17th, or worker warp 0) then
    // waits for `ready`, issues the pass from one lane and commits it to
    // `done`, on which the workers wait before reading the result.  With two
    // buffers, tile i + 1 is prepared and its pass 1 runs while tile i's pass
    // 2 runs and is written out.  Every worker runs the same sequence of
    // barriers whatever happens to `ok`.
    const int64_t stride = gridDim.x;
    if (G::ISSUER_WARP && warp == kGemmThreads / 32) {
        for (int64_t i = 0, tile = blockIdx.x; tile < ntiles; ++i, tile += stride) {
            const int b = G::NBUF == 2 ? static_cast<int>(i & 1) : 0;
            for (int pass = 0; pass < 2; ++pass) {
                gemm_wait(&ready[b], ph_ready[b], ok);
                if (ok && lane == 0) {
                    tc_fence_after();
                    issue(b, gemm_desc(smem_u32(plane_hi(b))), gemm_desc(smem_u32(plane_lo(b))));
                }
                __syncwarp();
            }
        }
    }
    auto publish = [&](int b) {
        fence_proxy_async();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ready[b]);
        if (!G::ISSUER_WARP && warp == 0) {
            gemm_wait(&ready[b], ph_ready[b], ok);
            if (ok && lane == 0) {
                tc_fence_after();
                issue(b, gemm_desc(smem_u32(plane_hi(b))), gemm_desc(smem_u32(plane_lo(b))));
            }
            __syncwarp();
        }
    };
    // 16384 points, in halves (quarters 0-1 and 2-3 of the radix-4 stage's
    // output): pass 1 over quarters 0-1 runs while 2-3 are stored, pass 1
    // over 2-3 while the first half of its output is twiddled, and so on.
    // Tile i's halves of D use tensor-memory blocks 2i mod 3 and 2i + 1 mod 3,
    // so that pass 1 over the next tile's quarters 0-1 runs (in the third
    // block, from the first halves of the planes) while this tile's output
    // is read and staged.
    auto publish_half = [&](int hf, int blk) {
        fence_proxy_async();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ready[hf]);
        if (warp == 0) {
            gemm_wait(&ready[hf], ph_ready[hf], ok);
            if (ok && lane == 0) {
                tc_fence_after();
                issue_half(hf, blk);
            }
            __syncwarp();
        }
    };
    if constexpr (LOGN == 14) {
        int64_t tile = blockIdx.x;
        if (tile < ntiles) {
            load(tile);
            radix4();
            put_quarters(0, 0);
            publish_half(0, 0);
            put_quarters(0, 2);
            publish_half(1, 1);
            if (tile + stride < ntiles) load(tile + stride);
        }
        for (int i = 0; tile < ntiles; ++i, tile += stride) {
            const bool more = tile + stride < ntiles;
            const int blk_a = (2 * i) % 3, blk_b = (2 * i + 1) % 3, blk_next = (2 * i + 2) % 3;
            gemm_wait(&done[0], ph_done[0], ok);  // pass 1, quarters 0-1
            tc_fence_after();
            epi1(0, 0, blk_a);
            publish_half(0, blk_a);
            gemm_wait(&done[1], ph_done[1], ok);  // pass 1, quarters 2-3
            tc_fence_after();
            epi1(0, 1, blk_b);
            publish_half(1, blk_b);
            gemm_wait(&done[0], ph_done[0], ok);  // pass 2, first half: rows 0..127 free
            if (more) {
                radix4();
                put_quarters(0, 0);
                publish_half(0, blk_next);
            }
            gemm_wait(&done[1], ph_done[1], ok);  // pass 2, second half
            tc_fence_after();
            epi2(0, tile, blk_a, blk_b);
            if (more) {
                put_quarters(0, 2);
                publish_half(1, blk_a);  // block blk_a was read by epi2
                if (tile + 2 * stride < ntiles) load(tile + 2 * stride);
            }
        }
    }
    int64_t tile = LOGN == 14 || (G::ISSUER_WARP && warp == kGemmThreads / 32) ? ntiles : blockIdx.x;
    if (tile < ntiles) {
        load(tile);
        prep(0);
        publish(0);
        if (tile + stride < ntiles) load(tile + stride);
    }
    for (int64_t i = 0; tile < ntiles; ++i, tile += stride) {
        const int cur = G::NBUF == 2 ? static_cast<int>(i & 1) : 0;
        const bool more = tile + stride < ntiles;
        gemm_wait(&done[cur], ph_done[cur], ok);  // pass 1 of this tile
        tc_fence_after();
        epi1(cur);
        publish(cur);
        if (G::NBUF == 2 && more) {
            prep(cur ^ 1);
            publish(cur ^ 1);
            if (tile + 2 * stride < ntiles) load(tile + 2 * stride);
        }
        gemm_wait(&done[cur], ph_done[cur], ok);  // pass 2 of this tile
        tc_fence_after();
        epi2(cur, tile);
        if (G::NBUF == 1 && more) {
            prep(0);
            publish(0);  // also releases the slot read by epi2
            if (tile + 2 * stride < ntiles) load(tile + 2 * stride);
        }
    }

    tc_fence_before();
    __syncthreads();
    // a product still in flight after a timeout lands before the tensor
    // memory is freed (bounded)
    if (!__syncthreads_and(ok) && tid == 0) {
#pragma unroll
        for (int b = 0; b < 2; ++b) mbar_wait_bounded(&done[b], ph_done[b]);
    }
    if (warp == 0) tmem_dealloc(tmem, kGemmTmemCols);
}

template <int PREC, int DIR>
const void *gemm_func_pd(int logn) {
    if (logn == 12) return reinterpret_cast<const void *>(&fft_tc_gemm_kernel<PREC, DIR, 12>);
    if (logn == 14) return reinterpret_cast<const void *>(&fft_tc_gemm_kernel<PREC, DIR, 14>);
    return nullptr;
}

}  // namespace

const void *fft_tc_gemm_func(int prec, int dir, int logn) {
    if (prec == BPLG_TC_BF16) return dir < 0 ? gemm_func_pd<BPLG_TC_BF16, -1>(logn) : gemm_func_pd<BPLG_TC_BF16, 1>(logn);
    if (prec == BPLG_TC_F16) return dir < 0 ? gemm_func_pd<BPLG_TC_F16, -1>(logn) : gemm_func_pd<BPLG_TC_F16, 1>(logn);
    return nullptr;
}

int fft_tc_gemm_smem(int logn) { return logn == 12 ? gemm_smem_bytes<12>() : gemm_smem_bytes<14>(); }

int fft_tc_gemm_threads(int logn) { return logn == 12 ? GemmShape<12>::BLOCK : GemmShape<14>::BLOCK; }

// persistent launch: one block per SM at most, tiles of two 4096-point
// signals or one 16384-point signal
int fft_tc_gemm_launch(const void *func, const void *in, void *out, int64_t n, int64_t batch, cudaStream_t s) {
    const int logn = ilog2(n);
    const int smem = fft_tc_gemm_smem(logn);
    int rc = ensure_smem_attr(func, smem);
    if (rc != BPLG_OK) return rc;
    const void *tw = nullptr;
    rc = twiddles_for_current_device(&tw);
    if (rc != BPLG_OK) return rc;
    const int64_t ntiles = logn == 12 ? (batch + 1) / 2 : batch;
    int64_t grid = 0;
    const int threads = fft_tc_gemm_threads(logn);
    rc = persistent_grid(func, threads, smem, ntiles, &grid);
    if (rc != BPLG_OK) return rc;
    void *args[] = {(void *)&in, (void *)&out, (void *)&tw, &batch};
    cudaError_t e = cudaLaunchKernel(func, dim3(static_cast<unsigned>(grid)), dim3(threads), args,
                                     static_cast<size_t>(smem), s);
    return e == cudaSuccess ? BPLG_OK : launch_error(e, "fft tc (two GEMM passes) launch", func, grid, threads, smem);
}

// Read (and optionally clear) the device error word of this file's kernel
// (its bounded waits on the MMA barrier) on the current device.
int fft_tc_gemm_device_status(int *flag, bool reset) {
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
