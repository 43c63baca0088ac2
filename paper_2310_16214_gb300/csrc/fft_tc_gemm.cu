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
// Fl Dh + Fh Dl + Fh Dh, accumulated in float32 in tensor memory:
//   pass 1: D1 = F x B1, B1 = the data (N = 64 columns per sub-signal,
//           K = [re n2 | im n2]); D1 row (k2, part), column (sub-signal, n1)
//   pass 2: D2 = A2 x F^T, A2 = the twiddled pass-1 output (rows (sub-signal,
//           k2), K = [re n1 | im n1]); D2 row (sub-signal, k2), column
//           (k1, part)
// One copy of F in shared memory (K-major, 16-byte core matrices without
// swizzle) serves as A in pass 1 and as B in pass 2.  Between the passes
// each thread reads one row of D1 from tensor memory, swaps halves with its
// neighbour lane (rows 2k2 and 2k2 + 1 hold the real and imaginary parts),
// applies the twiddles in float32 from the float64-generated table, splits
// and writes its row of A2.  D2 rows are read back with real and imaginary
// parts side by side, and a warp's lanes hold consecutive outputs, so the
// results go to global memory in 256-byte runs.
//
// Blocks are persistent (one per SM, 512 threads, 128 or 192 KB of shared
// memory) and load the next tile -- two 4096-point signals or one
// 16384-point signal -- into registers while the tensor cores run the
// current one.  Waits on the MMA barrier are bounded: on a timeout the block
// records the device error word and stops.
#include "device_util.cuh"
#include "fft_common.cuh"
#include "internal.h"
#include "tc_split.cuh"
#include "tcgen05.cuh"

namespace bplg {

namespace {

constexpr int kGemmThreads = 512;
constexpr int kGemmK = 128;                     // real K of a 64-point DFT
constexpr uint32_t kGemmSbo = 2048;             // bytes between 8-row groups (K = 128)
constexpr int kGemmPlane = 128 * kGemmK * 2;    // one 16-bit plane of F (32 KB)

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
    static constexpr int SIG = LOGN == 12 ? 2 : 1;     // signals per tile
    static constexpr int COLS = LOGN == 12 ? 128 : 256;  // pass-1 columns = pass-2 rows
    static constexpr int EPT = LOGN == 12 ? 16 : 32;     // complex values each thread loads
    static constexpr int DATA = COLS * kGemmK * 2;       // one 16-bit plane of the data operand
};

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

// W_m^e = exp(DIR 2 pi i e / m) from the table of exp(-2 pi i e / m)
template <int DIR>
__device__ __forceinline__ float2 root(const float2 *__restrict__ tw, int m, int e) {
    float2 w = __ldg(tw + m + e);
    if (DIR > 0) w.y = -w.y;
    return w;
}

// issue the products of one pass on the calling thread: D (+)= A B^T over
// K = 128, 8 steps of K = 16, three split products each
template <int PREC>
__device__ __forceinline__ void gemm_pass(uint32_t d, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi, uint32_t b_lo,
                                          uint32_t idesc) {
#pragma unroll
    for (int ks = 0; ks < kGemmK / 16; ++ks) {
        const uint32_t k = static_cast<uint32_t>(ks) * 256;  // two 128-byte core matrices per step
        umma_f16(d, gemm_desc(a_lo + k), gemm_desc(b_hi + k), idesc, ks > 0 ? 1u : 0u);
        umma_f16(d, gemm_desc(a_hi + k), gemm_desc(b_lo + k), idesc, 1u);
        umma_f16(d, gemm_desc(a_hi + k), gemm_desc(b_hi + k), idesc, 1u);
    }
}

// all threads: wait for the commit of the MMAs issued before; false (every
// thread) if the bounded wait ran out
__device__ __forceinline__ bool gemm_wait(uint64_t *bar, uint32_t &phase) {
    bool arrived = true;
    if (threadIdx.x < 32) arrived = mbar_wait_bounded(bar, phase);
    const bool ok = __syncthreads_and(arrived) != 0;
    phase ^= 1u;
    tc_fence_after();
    return ok;
}

template <int PREC, int DIR, int LOGN>
__global__ void __launch_bounds__(kGemmThreads, 1)
    fft_tc_gemm_kernel(const float2 *__restrict__ in, float2 *__restrict__ out, const float2 *__restrict__ tw,
                       int64_t batch) {
    using G = GemmShape<LOGN>;
    constexpr int N = 1 << LOGN;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *f_hi = smem;
    unsigned char *f_lo = smem + kGemmPlane;
    unsigned char *d_hi = smem + 2 * kGemmPlane;
    unsigned char *d_lo = d_hi + G::DATA;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t ntiles = (batch + G::SIG - 1) / G::SIG;

    if (warp == 0) {
        tmem_alloc(&tmem_slot, G::COLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    // F: row r = 2k + part_out, K column c = 64 part_in + n; W = exp(DIR 2 pi i k n / 64)
    for (int e = tid; e < 128 * 64; e += kGemmThreads) {
        const int r = e >> 6, c = (e & 63) * 2;
        float v[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = r >> 1, po = r & 1, pi = (c + h) >> 6, n = (c + h) & 63;
            const float2 w = root<DIR>(tw, 64, (k * n) & 63);
            v[h] = po == 0 ? (pi == 0 ? w.x : -w.y) : (pi == 0 ? w.y : w.x);
        }
        uint32_t hi, lo;
        HiLo<PREC>::pack(v[0], v[1], hi, lo);
        *reinterpret_cast<uint32_t *>(f_hi + gemm_off(r, c)) = hi;
        *reinterpret_cast<uint32_t *>(f_lo + gemm_off(r, c)) = lo;
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t sf_hi = smem_u32(f_hi), sf_lo = smem_u32(f_lo);
    const uint32_t sd_hi = smem_u32(d_hi), sd_lo = smem_u32(d_lo);
    const uint32_t tq = static_cast<uint32_t>(32 * (warp & 3)) << 16;  // this warp's tensor-memory lanes
    uint32_t phase = 0;
    bool ok = true;

    // thread -> (sub-signal or quarter, n1, n2 range) of the load
    const int n1 = tid & 63;
    float2 v[G::EPT];
    auto load = [&](int64_t tile) {
        if constexpr (LOGN == 12) {
            const int u = tid >> 8, q = (tid >> 6) & 3;
            const int64_t sig = tile * 2 + u;
            const float2 *src = in + sig * N + n1 + 64 * 16 * q;
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = sig < batch ? __ldcs(src + 64 * i) : make_float2(0.f, 0.f);
        } else {
            const int g = tid >> 6;
            const float2 *src = in + tile * N + n1 + 64 * 8 * g;
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) v[4 * i + q] = __ldcs(src + 64 * i + 4096 * q);
        }
    };

    int64_t tile = blockIdx.x;
    if (tile < ntiles) load(tile);
    for (; tile < ntiles && ok; tile += gridDim.x) {
        // ---- pass-1 operand: column (sub-signal, n1), K = [re n2 | im n2]
        if constexpr (LOGN == 12) {
            const int u = tid >> 8, q = (tid >> 6) & 3;
            const int row = u * 64 + n1;
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                float re[8], im[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    re[t] = v[8 * cc + t].x;
                    im[t] = v[8 * cc + t].y;
                }
                put_chunk<PREC>(d_hi, d_lo, gemm_off(row, 16 * q + 8 * cc), re);
                put_chunk<PREC>(d_hi, d_lo, gemm_off(row, 64 + 16 * q + 8 * cc), im);
            }
        } else {
            // radix-4 first stage, two n2 at a time (few live registers), each
            // output pair stored as one 32-bit word per plane
            const int g = tid >> 6;
#pragma unroll
            for (int i = 0; i < 8; i += 2) {
                float2 y[4][2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float2 a0 = v[4 * (i + h)], a1 = v[4 * (i + h) + 1];
                    const float2 a2 = v[4 * (i + h) + 2], a3 = v[4 * (i + h) + 3];
                    const float2 s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = csub(a1, a3);
                    // DIR i (a1 - a3)
                    const float2 jd = DIR < 0 ? make_float2(d13.y, -d13.x) : make_float2(-d13.y, d13.x);
                    const int k = n1 + 64 * (8 * g + i + h);
                    y[0][h] = cadd(s02, s13);
                    y[1][h] = cmul(cadd(d02, jd), root<DIR>(tw, 16384, k));
                    y[2][h] = cmul(csub(s02, s13), root<DIR>(tw, 16384, (2 * k) & 16383));
                    y[3][h] = cmul(csub(d02, jd), root<DIR>(tw, 16384, (3 * k) & 16383));
                }
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    uint32_t hr, lr, hi, li;
                    HiLo<PREC>::pack(y[m][0].x, y[m][1].x, hr, lr);
                    HiLo<PREC>::pack(y[m][0].y, y[m][1].y, hi, li);
                    const uint32_t ore = gemm_off(m * 64 + n1, 8 * g + i), oim = gemm_off(m * 64 + n1, 64 + 8 * g + i);
                    *reinterpret_cast<uint32_t *>(d_hi + ore) = hr;
                    *reinterpret_cast<uint32_t *>(d_lo + ore) = lr;
                    *reinterpret_cast<uint32_t *>(d_hi + oim) = hi;
                    *reinterpret_cast<uint32_t *>(d_lo + oim) = li;
                }
            }
        }
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            gemm_pass<PREC>(tmem, sf_hi, sf_lo, sd_hi, sd_lo, umma_idesc_f16(HiLo<PREC>::kFmt, 128, G::COLS));
            umma_commit(&bar);
        }
        // the next tile's loads are in flight while the tensor cores work
        if (tile + gridDim.x < ntiles) load(tile + gridDim.x);
        if (!gemm_wait(&bar, phase)) {
            ok = false;
            break;
        }

        // ---- D1 row (k2, part), columns (sub-signal, n1) -> twiddled A2 rows
        {
            const int r = 32 * (warp & 3) + lane;  // D1 row of this thread
            const int k2 = r >> 1, odd = r & 1;
            constexpr int CPW = G::COLS / 4;  // columns per warp: each lane quarter is read by 4 warps
            const int c0 = CPW * (warp >> 2);
#pragma unroll
            for (int h = 0; h < CPW / 16; ++h) {
                const int cb = c0 + 16 * h;  // 16 columns of one sub-signal
                uint32_t raw[16];
                tmem_ld16(tmem + tq + static_cast<uint32_t>(cb), raw);
                tmem_wait_ld();
                const int u = cb >> 6;
                const int nb = (cb & 63) + 8 * odd;  // this thread keeps n1 = nb .. nb + 7
                float re[8], im[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const uint32_t send = odd ? raw[t] : raw[8 + t];
                    const float got = __uint_as_float(__shfl_xor_sync(kFullMask, send, 1));
                    const float2 z = odd ? make_float2(got, __uint_as_float(raw[8 + t]))
                                         : make_float2(__uint_as_float(raw[t]), got);
                    const float2 zt = cmul(z, root<DIR>(tw, 4096, ((nb + t) * k2) & 4095));
                    re[t] = zt.x;
                    im[t] = zt.y;
                }
                int row;
                if constexpr (LOGN == 12)
                    row = u * 64 + k2;
                else
                    row = 128 * (k2 >> 5) + 4 * (k2 & 31) + u;
                put_chunk<PREC>(d_hi, d_lo, gemm_off(row, nb), re);
                put_chunk<PREC>(d_hi, d_lo, gemm_off(row, 64 + nb), im);
            }
        }
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int hh = 0; hh < G::COLS / 128; ++hh) {
                const uint32_t a = static_cast<uint32_t>(hh) * 16 * kGemmSbo;  // rows 128 hh ..
                gemm_pass<PREC>(tmem + static_cast<uint32_t>(128 * hh), sd_hi + a, sd_lo + a, sf_hi, sf_lo,
                                umma_idesc_f16(HiLo<PREC>::kFmt, 128, 128));
            }
            umma_commit(&bar);
        }
        if (!gemm_wait(&bar, phase)) {
            ok = false;
            break;
        }

        // ---- D2 row (sub-signal, k2), columns (k1, part) -> X
        {
            const int r = 32 * (warp & 3) + lane;
            constexpr int CPW = G::COLS / 4;
            const int c0 = CPW * (warp >> 2);
#pragma unroll
            for (int h = 0; h < CPW / 16; ++h) {
                const int cb = c0 + 16 * h;
                uint32_t raw[16];
                tmem_ld16(tmem + tq + static_cast<uint32_t>(cb), raw);
                tmem_wait_ld();
                const int hh = cb >> 7;
                const int k1b = (cb & 127) >> 1;  // eight outputs k1 = k1b .. k1b + 7
                if constexpr (LOGN == 12) {
                    const int u = r >> 6, k2 = r & 63;
                    const int64_t sig = tile * 2 + u;
                    if (sig < batch) {
                        float2 *dst = out + sig * N + k2 + 64 * k1b;
#pragma unroll
                        for (int t = 0; t < 8; ++t)
                            __stcs(dst + 64 * t, make_float2(__uint_as_float(raw[2 * t]), __uint_as_float(raw[2 * t + 1])));
                    }
                } else {
                    // X[4 (k2 + 64 k1) + u] with u = r & 3, k2 = 32 hh + r / 4: lanes consecutive
                    float2 *dst = out + tile * N + 128 * hh + r + 256 * k1b;
#pragma unroll
                    for (int t = 0; t < 8; ++t)
                        __stcs(dst + 256 * t, make_float2(__uint_as_float(raw[2 * t]), __uint_as_float(raw[2 * t + 1])));
                }
            }
        }
        tc_fence_before();
        __syncthreads();  // tensor memory and the data planes are free for the next tile
    }

    tc_fence_before();
    __syncthreads();
    if (!ok && tid == 0) mbar_wait_bounded(&bar, phase);  // let a late commit land before freeing
    if (warp == 0) tmem_dealloc(tmem, G::COLS);
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

// F (two planes) and the data operand (two planes)
int fft_tc_gemm_smem(int logn) {
    return 2 * kGemmPlane + 2 * (logn == 12 ? GemmShape<12>::DATA : GemmShape<14>::DATA);
}

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
    rc = persistent_grid(func, kGemmThreads, smem, ntiles, &grid);
    if (rc != BPLG_OK) return rc;
    void *args[] = {(void *)&in, (void *)&out, (void *)&tw, &batch};
    cudaError_t e = cudaLaunchKernel(func, dim3(static_cast<unsigned>(grid)), dim3(kGemmThreads), args,
                                     static_cast<size_t>(smem), s);
    return e == cudaSuccess ? BPLG_OK : launch_error(e, "fft tc (two GEMM passes) launch", func, grid, kGemmThreads, smem);
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
