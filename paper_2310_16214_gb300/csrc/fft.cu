// Batched complex Stockham FFT (Section III, "Fast Fourier Transform",
// Fig. 1(c); knobs of Section V-C).
//
// A block holds `spb` signals of n = 2^logn points; each signal is served by
// T = n/R threads and every thread computes one radix-R butterfly per stage
// (P = r, as in the paper).  Stage s (stride Ns = product of the earlier
// radices) reads x[j + m T], m = 0..R-1, multiplies element m by W_{Ns R}^{m k}
// with k = j mod Ns, runs an R-point DFT in registers and writes element r to
// (j div Ns) Ns R + k + r Ns -- the self-sorting Stockham index map, so the
// result comes out in natural order with no bit reversal.  When log2 R does
// not divide logn the first stage uses the lower radix 2^(logn mod log2 R)
// (the mixed-radix technique of Section VI-A), each thread then doing R/R0
// butterflies.  Stages exchange data through shared memory:
//   smem_layout 0  interleaved complex, one float2 per element;
//   smem_layout 1  real parts then imaginary parts through one float buffer
//                  (the exchange multiplexing of Section V-C: half the space);
//   smem_pad       one pad slot per 16 (float2) or 32 (float) elements, which
//                  makes the strided Stockham writes conflict-free;
//   io 0 / 1       first and last stage talk to global memory directly
//                  (8-byte coalesced), or the whole tile is staged through
//                  shared memory with 16-byte accesses.
// Twiddles W_M^k = exp(-2 pi i k / M) are generated once per device in float64
// (sincospi) and rounded to float32; the inverse uses their conjugates.
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "device_util.cuh"
#include "internal.h"
#include "fft_common.cuh"
#include "tma.cuh"

namespace bplg {

// size-specialised kernels (fft_fixed_fwd.cu / fft_fixed_inv.cu); nullptr
// when (radix, layout, threads, log2 n) has no instantiation
const void *fft_fixed_lookup_fwd(int radix, int layout, int threads, int logn);
const void *fft_fixed_lookup_inv(int radix, int layout, int threads, int logn);

template <int R, int DIR, int LAYOUT, int PAD, int STAGED, int MAXT>
__global__ void __launch_bounds__(MAXT)
    fft_kernel(const float2 *in, float2 *out, const float2 *__restrict__ tw, int logn, int spb,
               int64_t batch) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int LR = clog2(R);
    const int n = 1 << logn;
    const int logT = logn - LR;
    const int T = 1 << logT;
    const int tid = threadIdx.x;
    const int s = tid >> logT;
    const int j = tid & (T - 1);
    const int64_t sig0 = static_cast<int64_t>(blockIdx.x) * spb;
    const int64_t sig = sig0 + s;
    const bool active = sig < batch;
    const int64_t left = batch - sig0;
    const int nvalid = left < spb ? static_cast<int>(left) : spb;
    const int stride = sig_stride<LAYOUT, PAD>(n);
    float2 *buf2 = reinterpret_cast<float2 *>(smem_raw);
    float *buf1 = reinterpret_cast<float *>(smem_raw);
    const int sbase = s * stride;

    float2 v[R];
    OutMap om{0, 0, 0, 0, 0, j, T};
    if constexpr (STAGED) {
        const float4 *g = reinterpret_cast<const float4 *>(in + sig0 * n);
        const int count4 = (nvalid * n) >> 1;
        for (int q = tid; q < count4; q += blockDim.x) {
            float4 w = __ldcs(g + q);
            const int e0 = q << 1;
            const int ss = e0 >> logn;
            const int e = e0 & (n - 1);
            buf2[ss * stride + pidx<0, PAD>(e)] = make_float2(w.x, w.y);
            buf2[ss * stride + pidx<0, PAD>(e + 1)] = make_float2(w.z, w.w);
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = buf2[sbase + pidx<0, PAD>(j + m * T)];
    } else {
        const float2 *g = in + sig * n + j;
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = active ? __ldcs(g + m * T) : make_float2(0.f, 0.f);
    }

    const int lr0 = logn % LR;
    const int nstages = (lr0 ? 1 : 0) + logn / LR;
    int logNs = 0;
    for (int st = 0; st < nstages; ++st) {
        if (st == 0 && lr0 != 0) {
            if constexpr (R >= 4) {
                if (lr0 == 1) first_stage_mixed<R, 2, DIR>(v);
            }
            if constexpr (R >= 8) {
                if (lr0 == 2) first_stage_mixed<R, 4, DIR>(v);
            }
            if constexpr (R >= 16) {
                if (lr0 == 3) first_stage_mixed<R, 8, DIR>(v);
            }
            om.mixed = 1;
            om.lr0 = lr0;
            om.lq = LR - lr0;
            logNs = lr0;
        } else {
            const int Ns = 1 << logNs;
            const int k = j & (Ns - 1);
            if (logNs > 0) {
                const float2 *twp = tw + (Ns << LR);
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    float2 w = __ldg(twp + r * k);
                    if (DIR > 0) w.y = -w.y;
                    v[r] = cmul(v[r], w);
                }
            }
            dft_codelet<R, DIR>(v);
            om.mixed = 0;
            om.base = ((j >> logNs) << (logNs + LR)) + k;
            om.shift = logNs;
            logNs += LR;
        }
        if (st == nstages - 1) break;
        // exchange through shared memory for the next stage
        if constexpr (LAYOUT == 0) {
            __syncthreads();
#pragma unroll
            for (int r = 0; r < R; ++r) buf2[sbase + pidx<0, PAD>(om(r))] = v[r];
            __syncthreads();
#pragma unroll
            for (int m = 0; m < R; ++m) v[m] = buf2[sbase + pidx<0, PAD>(j + m * T)];
        } else {
            __syncthreads();
#pragma unroll
            for (int r = 0; r < R; ++r) buf1[sbase + pidx<1, PAD>(om(r))] = v[r].x;
            __syncthreads();
#pragma unroll
            for (int m = 0; m < R; ++m) v[m].x = buf1[sbase + pidx<1, PAD>(j + m * T)];
            __syncthreads();
#pragma unroll
            for (int r = 0; r < R; ++r) buf1[sbase + pidx<1, PAD>(om(r))] = v[r].y;
            __syncthreads();
#pragma unroll
            for (int m = 0; m < R; ++m) v[m].y = buf1[sbase + pidx<1, PAD>(j + m * T)];
        }
    }

    if constexpr (STAGED) {
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R; ++r) buf2[sbase + pidx<0, PAD>(om(r))] = v[r];
        __syncthreads();
        float4 *g = reinterpret_cast<float4 *>(out + sig0 * n);
        const int count4 = (nvalid * n) >> 1;
        for (int q = tid; q < count4; q += blockDim.x) {
            const int e0 = q << 1;
            const int ss = e0 >> logn;
            const int e = e0 & (n - 1);
            float2 lo = buf2[ss * stride + pidx<0, PAD>(e)];
            float2 hi = buf2[ss * stride + pidx<0, PAD>(e + 1)];
            __stcs(g + q, make_float4(lo.x, lo.y, hi.x, hi.y));
        }
    } else {
        if (active) {
            float2 *g = out + sig * n;
#pragma unroll
            for (int r = 0; r < R; ++r) __stcs(g + om(r), v[r]);
        }
    }
}

// Persistent, TMA-pipelined variant (io = 2).  Grid = the resident-block
// capacity of the device; each block walks tiles (spb consecutive signals)
// tile = blockIdx.x, blockIdx.x + gridDim.x, ...  A ring of NS shared-memory
// slots holds the tiles: one bulk asynchronous copy (cp.async.bulk) per tile,
// completion tracked by one mbarrier per slot, so while a tile is computed
// the next NS-1 tiles are already streaming in.  With T >= 32 threads per
// signal the first stage reads the slot directly (consecutive lanes,
// conflict-free), the stage exchanges reuse the slot with the padded layout,
// and the last stage stores straight to global memory (coalesced).  With
// T < 32 the tile is first re-laid into a padded exchange buffer and written
// back through it with 16-byte stores.  Waits are bounded: on timeout the
// block records an error, drains its own copies (bounded) and returns.
template <int R, int DIR, int PAD, int MAXT, int NS>
__global__ void __launch_bounds__(MAXT)
    fft_tma_kernel(const float2 *in, float2 *out, const float2 *__restrict__ tw, int logn, int spb, int64_t batch,
                   int64_t ntiles, int slot_elems) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[NS];
    constexpr int LR = clog2(R);
    const int n = 1 << logn;
    const int logT = logn - LR;
    const int T = 1 << logT;
    const int tid = threadIdx.x;
    const int s = tid >> logT;
    const int j = tid & (T - 1);
    const int stride = sig_stride<0, PAD>(n);
    const bool small = T < 32;
    float2 *slots = reinterpret_cast<float2 *>(smem_raw);
    float2 *xbuf = slots + static_cast<size_t>(NS) * slot_elems;
    const int sbase = s * stride;
    // issuer state (thread 0 only): loads issued / consumed per slot
    int issued[NS], consumed[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) issued[q] = consumed[q] = 0;

    auto issue = [&](int64_t tile, int q) {
        const int64_t sig0 = tile * spb;
        const int64_t left = batch - sig0;
        const int nv = left < spb ? static_cast<int>(left) : spb;
        const uint32_t bytes = static_cast<uint32_t>(nv) * static_cast<uint32_t>(n) * 8u;
        mbar_arrive_expect_tx(&full[q], bytes);
        tma_load_1d(slots + static_cast<size_t>(q) * slot_elems, in + sig0 * n, bytes, &full[q]);
        ++issued[q];
    };

    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NS; ++q) mbar_init(&full[q], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            const int64_t tile = blockIdx.x + static_cast<int64_t>(q) * gridDim.x;
            if (tile < ntiles) issue(tile, q);
        }
    }

    int k = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
        const int q = k % NS;
        const uint32_t parity = static_cast<uint32_t>(k / NS) & 1u;
        float2 *slot = slots + static_cast<size_t>(q) * slot_elems;
        const int64_t sig0 = tile * spb;
        const int64_t left = batch - sig0;
        const int nvalid = left < spb ? static_cast<int>(left) : spb;
        const bool active = s < nvalid;
        const bool ok = __syncthreads_and(mbar_wait_bounded(&full[q], parity));
        if (!ok) {
            if (tid == 0) {  // drain this block's copies in flight, then leave
#pragma unroll
                for (int qq = 0; qq < NS; ++qq)
                    if (issued[qq] > consumed[qq]) mbar_wait_bounded(&full[qq], static_cast<uint32_t>(consumed[qq]) & 1u);
            }
            return;
        }
        if (tid == 0) ++consumed[q];
        const int64_t next = tile + static_cast<int64_t>(NS) * gridDim.x;

        float2 v[R];
        OutMap om{0, 0, 0, 0, 0, j, T};
        float2 *ex;
        if (!small) {
#pragma unroll
            for (int m = 0; m < R; ++m) v[m] = slot[s * n + j + m * T];
            ex = slot;
        } else {
            const int count4 = (nvalid * n) >> 1;
            const float4 *src = reinterpret_cast<const float4 *>(slot);
            for (int qq = tid; qq < count4; qq += blockDim.x) {
                const float4 w = src[qq];
                const int e0 = qq << 1;
                const int ss = e0 >> logn;
                const int e = e0 & (n - 1);
                xbuf[ss * stride + pidx<0, PAD>(e)] = make_float2(w.x, w.y);
                xbuf[ss * stride + pidx<0, PAD>(e + 1)] = make_float2(w.z, w.w);
            }
            __syncthreads();
            if (tid == 0 && next < ntiles) {
                fence_proxy_async();
                issue(next, q);
            }
#pragma unroll
            for (int m = 0; m < R; ++m) v[m] = xbuf[sbase + pidx<0, PAD>(j + m * T)];
            ex = xbuf;
        }

        const int lr0 = logn % LR;
        const int nstages = (lr0 ? 1 : 0) + logn / LR;
        int logNs = 0;
        for (int st = 0; st < nstages; ++st) {
            if (st == 0 && lr0 != 0) {
                if constexpr (R >= 4) {
                    if (lr0 == 1) first_stage_mixed<R, 2, DIR>(v);
                }
                if constexpr (R >= 8) {
                    if (lr0 == 2) first_stage_mixed<R, 4, DIR>(v);
                }
                if constexpr (R >= 16) {
                    if (lr0 == 3) first_stage_mixed<R, 8, DIR>(v);
                }
                om.mixed = 1;
                om.lr0 = lr0;
                om.lq = LR - lr0;
                logNs = lr0;
            } else {
                const int Ns = 1 << logNs;
                const int kk = j & (Ns - 1);
                if (logNs > 0) {
                    const float2 *twp = tw + (Ns << LR);
#pragma unroll
                    for (int r = 1; r < R; ++r) {
                        float2 w = __ldg(twp + r * kk);
                        if (DIR > 0) w.y = -w.y;
                        v[r] = cmul(v[r], w);
                    }
                }
                dft_codelet<R, DIR>(v);
                om.mixed = 0;
                om.base = ((j >> logNs) << (logNs + LR)) + kk;
                om.shift = logNs;
                logNs += LR;
            }
            if (st == nstages - 1) break;
            __syncthreads();
#pragma unroll
            for (int r = 0; r < R; ++r) ex[sbase + pidx<0, PAD>(om(r))] = v[r];
            __syncthreads();
#pragma unroll
            for (int m = 0; m < R; ++m) v[m] = ex[sbase + pidx<0, PAD>(j + m * T)];
        }

        if (!small) {
            if (active) {
                float2 *g = out + (sig0 + s) * n;
#pragma unroll
                for (int r = 0; r < R; ++r) __stcs(g + om(r), v[r]);
            }
            __syncthreads();  // every read of the slot is done: refill it
            if (tid == 0 && next < ntiles) {
                fence_proxy_async();
                issue(next, q);
            }
        } else {
            __syncthreads();
#pragma unroll
            for (int r = 0; r < R; ++r) xbuf[sbase + pidx<0, PAD>(om(r))] = v[r];
            __syncthreads();
            float4 *g = reinterpret_cast<float4 *>(out + sig0 * n);
            const int count4 = (nvalid * n) >> 1;
            for (int qq = tid; qq < count4; qq += blockDim.x) {
                const int e0 = qq << 1;
                const int ss = e0 >> logn;
                const int e = e0 & (n - 1);
                const float2 lo = xbuf[ss * stride + pidx<0, PAD>(e)];
                const float2 hi = xbuf[ss * stride + pidx<0, PAD>(e + 1)];
                __stcs(g + qq, make_float4(lo.x, lo.y, hi.x, hi.y));
            }
            __syncthreads();  // xbuf is rewritten by the next tile
        }
    }
}

constexpr int kFftTmaStages = 3;

// The pipelined variant with the compile-time stage schedule: radix 16,
// padded exchanges, n = 2^LOGN >= 512 (T >= 32, so the first stage reads the
// ring slot directly and the last stage stores straight to global memory).
// The ring, the bounded waits and the refill protocol are those of
// fft_tma_kernel.
template <int LOGN, int DIR, int MAXT, int NS>
__global__ void __launch_bounds__(MAXT)
    fft_tma_fixed_kernel(const float2 *in, float2 *out, const float2 *__restrict__ tw, int logn, int spb,
                         int64_t batch, int64_t ntiles, int slot_elems) {
    using S = FftShape<16, LOGN>;
    static_assert(S::T >= 32, "the slot is read directly only with T >= 32");
    constexpr int N = 1 << LOGN;
    constexpr int STRIDE = N + N / 16;
    (void)logn;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[NS];
    const int tid = threadIdx.x;
    const int s = tid >> S::LOGT;
    const int j = tid & (S::T - 1);
    float2 *slots = reinterpret_cast<float2 *>(smem_raw);
    int issued[NS], consumed[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) issued[q] = consumed[q] = 0;

    auto issue = [&](int64_t tile, int q) {
        const int64_t sig0 = tile * spb;
        const int64_t left = batch - sig0;
        const int nv = left < spb ? static_cast<int>(left) : spb;
        const uint32_t bytes = static_cast<uint32_t>(nv) * static_cast<uint32_t>(N) * 8u;
        mbar_arrive_expect_tx(&full[q], bytes);
        tma_load_1d(slots + static_cast<size_t>(q) * slot_elems, in + sig0 * N, bytes, &full[q]);
        ++issued[q];
    };

    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NS; ++q) mbar_init(&full[q], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            const int64_t tile = blockIdx.x + static_cast<int64_t>(q) * gridDim.x;
            if (tile < ntiles) issue(tile, q);
        }
    }

    int k = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
        const int q = k % NS;
        const uint32_t parity = static_cast<uint32_t>(k / NS) & 1u;
        float2 *slot = slots + static_cast<size_t>(q) * slot_elems;
        const int64_t sig0 = tile * spb;
        const bool active = sig0 + s < batch;
        const bool ok = __syncthreads_and(mbar_wait_bounded(&full[q], parity));
        if (!ok) {
            if (tid == 0) {  // drain this block's copies in flight, then leave
#pragma unroll
                for (int qq = 0; qq < NS; ++qq)
                    if (issued[qq] > consumed[qq]) mbar_wait_bounded(&full[qq], static_cast<uint32_t>(consumed[qq]) & 1u);
            }
            return;
        }
        if (tid == 0) ++consumed[q];
        float2 v[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = slot[s * N + j + m * S::T];
        fft_fixed_stages<16, LOGN, DIR, 0, 0>(v, slot + s * STRIDE, nullptr, j, tw, out + (sig0 + s) * N, active);
        __syncthreads();  // every read of the slot is done: refill it
        const int64_t next = tile + static_cast<int64_t>(NS) * gridDim.x;
        if (tid == 0 && next < ntiles) {
            fence_proxy_async();
            issue(next, q);
        }
    }
}

// Split-exchange pipelined variant (io 2 with smem_layout 1): radix 16,
// n = 2^LOGN >= 1024.  The ring slots hold the tiles unpadded; the stage
// exchanges go through a separate real/imaginary float buffer (the
// multiplexed layout), so a slot is free as soon as the first stage has read
// it and its refill starts right away, overlapping the rest of the tile's
// stages.  This is what lets a transform that needs a whole SM per signal
// (n = 16384: 1024 threads, one block per SM) keep a load in flight.
template <int LOGN>
struct SplitRing {
    // One slot: it is refilled as soon as the first stage has read it, so
    // the next tile's copy already overlaps the remaining stages, and the
    // block keeps the shared-memory footprint (and occupancy) of a single
    // tile plus its exchange buffer.
    static constexpr int NS = 1;
};

template <int LOGN, int DIR, int MAXT>
__global__ void __launch_bounds__(MAXT)
    fft_tma_split_kernel(const float2 *in, float2 *out, const float2 *__restrict__ tw, int logn, int spb,
                         int64_t batch, int64_t ntiles, int slot_elems) {
    using S = FftShape<16, LOGN>;
    constexpr int NS = SplitRing<LOGN>::NS;
    constexpr int N = 1 << LOGN;
    constexpr int STRIDE1 = N + N / 32;  // floats per signal in the exchange buffer
    (void)logn;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[NS];
    const int tid = threadIdx.x;
    const int s = tid >> S::LOGT;
    const int j = tid & (S::T - 1);
    float2 *slots = reinterpret_cast<float2 *>(smem_raw);
    float *xbuf = reinterpret_cast<float *>(slots + static_cast<size_t>(NS) * slot_elems) + s * STRIDE1;
    int issued[NS], consumed[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) issued[q] = consumed[q] = 0;

    auto issue = [&](int64_t tile, int q) {
        const int64_t sig0 = tile * spb;
        const int64_t left = batch - sig0;
        const int nv = left < spb ? static_cast<int>(left) : spb;
        const uint32_t bytes = static_cast<uint32_t>(nv) * static_cast<uint32_t>(N) * 8u;
        mbar_arrive_expect_tx(&full[q], bytes);
        tma_load_1d(slots + static_cast<size_t>(q) * slot_elems, in + sig0 * N, bytes, &full[q]);
        ++issued[q];
    };

    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NS; ++q) mbar_init(&full[q], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            const int64_t tile = blockIdx.x + static_cast<int64_t>(q) * gridDim.x;
            if (tile < ntiles) issue(tile, q);
        }
    }

    int k = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
        const int q = k % NS;
        const uint32_t parity = static_cast<uint32_t>(k / NS) & 1u;
        const float2 *slot = slots + static_cast<size_t>(q) * slot_elems;
        const int64_t sig0 = tile * spb;
        const bool active = sig0 + s < batch;
        const bool ok = __syncthreads_and(mbar_wait_bounded(&full[q], parity));
        if (!ok) {
            if (tid == 0) {  // drain this block's copies in flight, then leave
#pragma unroll
                for (int qq = 0; qq < NS; ++qq)
                    if (issued[qq] > consumed[qq]) mbar_wait_bounded(&full[qq], static_cast<uint32_t>(consumed[qq]) & 1u);
            }
            return;
        }
        if (tid == 0) ++consumed[q];
        float2 v[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = slot[s * N + j + m * S::T];
        __syncthreads();  // every read of the slot is done: refill it now
        const int64_t next = tile + static_cast<int64_t>(NS) * gridDim.x;
        if (tid == 0 && next < ntiles) {
            fence_proxy_async();
            issue(next, q);
        }
        fft_fixed_stages<16, LOGN, DIR, 1, 0>(v, nullptr, xbuf, j, tw, out + (sig0 + s) * N, active);
    }
}

// Twiddle table: tw[M + k] = exp(-2 pi i k / M) for M = 2, 4, ..., 2^max_log,
// computed in float64 and rounded once to float32.
__global__ void twiddle_init_kernel(float2 *tw, int max_log) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t total = int64_t(2) << max_log;
    if (i >= total) return;
    if (i < 2) {
        tw[i] = make_float2(1.f, 0.f);
        return;
    }
    const int lm = 63 - __clzll(static_cast<unsigned long long>(i));
    const int64_t M = int64_t(1) << lm;
    const int64_t k = i - M;
    double sn, cs;
    sincospi(-2.0 * static_cast<double>(k) / static_cast<double>(M), &sn, &cs);
    tw[i] = make_float2(static_cast<float>(cs), static_cast<float>(sn));
}

namespace {

// Radix-16 butterflies need more than the 64 registers a 1024-thread block
// leaves per thread; blocks of at most 512 threads use an instantiation
// bounded to 512 threads (up to 128 registers).
template <int R, int DIR, int LAYOUT, int PAD, int MAXT>
const void *fft_func_io_t(int io) {
    if constexpr (LAYOUT == 1) {
        return io == 0 ? reinterpret_cast<const void *>(&fft_kernel<R, DIR, 1, PAD, 0, MAXT>) : nullptr;
    } else {
        if (io == 2) return reinterpret_cast<const void *>(&fft_tma_kernel<R, DIR, PAD, MAXT, kFftTmaStages>);
        return io == 0 ? reinterpret_cast<const void *>(&fft_kernel<R, DIR, 0, PAD, 0, MAXT>)
                       : reinterpret_cast<const void *>(&fft_kernel<R, DIR, 0, PAD, 1, MAXT>);
    }
}

template <int DIR, int MAXT>
const void *fft_tma_fixed_func(int logn) {
    switch (logn) {
        case 10: return reinterpret_cast<const void *>(&fft_tma_fixed_kernel<10, DIR, MAXT, kFftTmaStages>);
        case 11: return reinterpret_cast<const void *>(&fft_tma_fixed_kernel<11, DIR, MAXT, kFftTmaStages>);
        case 12: return reinterpret_cast<const void *>(&fft_tma_fixed_kernel<12, DIR, MAXT, kFftTmaStages>);
        case 13: return reinterpret_cast<const void *>(&fft_tma_fixed_kernel<13, DIR, MAXT, kFftTmaStages>);
        case 14: return reinterpret_cast<const void *>(&fft_tma_fixed_kernel<14, DIR, MAXT, kFftTmaStages>);
        default: return nullptr;
    }
}

template <int DIR, int MAXT>
const void *fft_tma_split_func(int logn) {
    switch (logn) {
        case 10: return reinterpret_cast<const void *>(&fft_tma_split_kernel<10, DIR, MAXT>);
        case 11: return reinterpret_cast<const void *>(&fft_tma_split_kernel<11, DIR, MAXT>);
        case 12: return reinterpret_cast<const void *>(&fft_tma_split_kernel<12, DIR, MAXT>);
        case 13: return reinterpret_cast<const void *>(&fft_tma_split_kernel<13, DIR, MAXT>);
        case 14: return reinterpret_cast<const void *>(&fft_tma_split_kernel<14, DIR, MAXT>);
        default: return nullptr;
    }
}

template <int R, int DIR, int LAYOUT, int PAD>
const void *fft_func_io(int io, int threads, int logn) {
    if constexpr ((R == 16 || R == 8) && PAD == 1) {
        if (io == 0) {
            const void *f = DIR < 0 ? fft_fixed_lookup_fwd(R, LAYOUT, threads, logn)
                                    : fft_fixed_lookup_inv(R, LAYOUT, threads, logn);
            if (f) return f;
        }
    }
    if constexpr (R == 16 && PAD == 1) {
        if (LAYOUT == 0 && io == 2 && logn >= 10 && logn <= 14)
            return threads <= 512 ? fft_tma_fixed_func<DIR, 512>(logn) : fft_tma_fixed_func<DIR, 1024>(logn);
        if (LAYOUT == 1 && io == 2 && logn >= 10 && logn <= 14)
            return threads <= 512 ? fft_tma_split_func<DIR, 512>(logn) : fft_tma_split_func<DIR, 1024>(logn);
    }
    if constexpr (R == 16) {
        if (threads <= 512) return fft_func_io_t<R, DIR, LAYOUT, PAD, 512>(io);
    }
    return fft_func_io_t<R, DIR, LAYOUT, PAD, 1024>(io);
}

template <int R, int DIR>
const void *fft_func_rd(int layout, int pad, int io, int threads, int logn) {
    if (layout == 0)
        return pad ? fft_func_io<R, DIR, 0, 1>(io, threads, logn) : fft_func_io<R, DIR, 0, 0>(io, threads, logn);
    return pad ? fft_func_io<R, DIR, 1, 1>(io, threads, logn) : fft_func_io<R, DIR, 1, 0>(io, threads, logn);
}

template <int DIR>
const void *fft_func_d(int radix, int layout, int pad, int io, int threads, int logn) {
    switch (radix) {
        case 2: return fft_func_rd<2, DIR>(layout, pad, io, threads, logn);
        case 4: return fft_func_rd<4, DIR>(layout, pad, io, threads, logn);
        case 8: return fft_func_rd<8, DIR>(layout, pad, io, threads, logn);
        case 16: return fft_func_rd<16, DIR>(layout, pad, io, threads, logn);
        default: return nullptr;
    }
}

const void *fft_func(int radix, int dir, int layout, int pad, int io, int threads, int logn) {
    if (layout < 0 || layout > 1 || pad < 0 || pad > 1 || io < 0 || io > 2) return nullptr;
    return dir < 0 ? fft_func_d<-1>(radix, layout, pad, io, threads, logn)
                   : fft_func_d<1>(radix, layout, pad, io, threads, logn);
}

std::mutex g_tw_mu;
std::unordered_map<int, float2 *> g_tw;

}  // namespace

// elements of one ring slot of the pipelined kernel (128-byte multiple)
int fft_tma_slot_elems(int pad, int64_t n, int spb);

// slots of the split-exchange ring: the tile unpadded
static int split_slots(int64_t n) {
    switch (ilog2(n)) {
        case 10: return SplitRing<10>::NS;
        case 11: return SplitRing<11>::NS;
        case 12: return SplitRing<12>::NS;
        case 13: return SplitRing<13>::NS;
        default: return SplitRing<14>::NS;
    }
}

int fft_tma_slot_elems_layout(int layout, int pad, int64_t n, int spb) {
    if (layout == 1) return static_cast<int>((static_cast<int64_t>(spb) * n + 15) & ~int64_t(15));
    return fft_tma_slot_elems(pad, n, spb);
}

int fft_tma_slot_elems(int pad, int64_t n, int spb) {
    const int logn = ilog2(n);
    (void)logn;
    const int64_t padded = static_cast<int64_t>(spb) * (pad ? sig_stride<0, 1>(static_cast<int>(n)) : static_cast<int>(n));
    return static_cast<int>((padded + 15) & ~int64_t(15));
}

int fft_smem_bytes(int radix, int layout, int pad, int io, int64_t n, int spb) {
    const int logn = ilog2(n);
    if (io == 2 && layout == 1) {  // split-exchange ring: slots + real/imaginary exchange buffer
        const int64_t slot = fft_tma_slot_elems_layout(1, pad, n, spb);
        return static_cast<int>(split_slots(n) * slot * 8 + static_cast<int64_t>(spb) * sig_stride<1, 1>(static_cast<int>(n)) * 4);
    }
    if (io == 2) {
        const int64_t T = n / radix;
        const int64_t slot = fft_tma_slot_elems(pad, n, spb);
        const int64_t xb = T < 32 ? static_cast<int64_t>(spb) * (pad ? sig_stride<0, 1>(static_cast<int>(n)) : n) : 0;
        return static_cast<int>((kFftTmaStages * slot + xb) * 8);
    }
    const int lr = ilog2(radix);
    const int nstages = (logn % lr ? 1 : 0) + logn / lr;
    if (nstages <= 1 && io == 0) return 0;
    const int stride = layout == 0 ? (pad ? sig_stride<0, 1>(static_cast<int>(n)) : static_cast<int>(n))
                                   : (pad ? sig_stride<1, 1>(static_cast<int>(n)) : static_cast<int>(n));
    return spb * stride * (layout == 0 ? 8 : 4);
}

int twiddles_for_current_device(const void **tw) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lock(g_tw_mu);
    auto it = g_tw.find(dev);
    if (it != g_tw.end()) {
        *tw = it->second;
        return BPLG_OK;
    }
    const int64_t total = int64_t(2) << kFftMaxLog;
    float2 *p = nullptr;
    e = cudaMalloc(&p, total * sizeof(float2));
    if (e != cudaSuccess) return cuda_error(e, "twiddle table cudaMalloc");
    cudaStream_t st;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaFree(p);
        return cuda_error(e, "twiddle stream");
    }
    twiddle_init_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, st>>>(p, kFftMaxLog);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (e != cudaSuccess) {
        cudaFree(p);
        return cuda_error(e, "twiddle generation");
    }
    g_tw[dev] = p;
    *tw = p;
    return BPLG_OK;
}

bool fft_launch_info(const bplg_plan &p, int64_t n, int64_t batch, int dir, Launch *out) {
    if (n > (int64_t(1) << kFftMaxLog)) return fft_large_launch_info(p, n, batch, dir, 0, out);
    std::string why;
    if (!plan_structurally_valid(p, BPLG_F32, n, &why)) return false;
    const void *f = fft_func(p.radix, dir, p.smem_layout, p.smem_pad, p.io, p.L, ilog2(n));
    if (!f) return false;
    out->func = f;
    out->threads = p.L;
    out->smem = fft_smem_bytes(p.radix, p.smem_layout, p.smem_pad, p.io, n, p.spb);
    out->blocks = (batch + p.spb - 1) / p.spb;
    return true;
}

int fft_launch(const bplg_plan &p, const void *in, void *out, int64_t n, int64_t batch, int dir,
               cudaStream_t s) {
    if (n > (int64_t(1) << kFftMaxLog)) return fft_large_launch(p, in, out, n, batch, dir, s);
    Launch li;
    if (!fft_launch_info(p, n, batch, dir, &li)) return set_error(BPLG_ERR_INVALID_PLAN, "fft: plan has no kernel");
    int rc = check_grid(li.blocks, "fft");
    if (rc != BPLG_OK) return rc;
    const void *tw = nullptr;
    rc = twiddles_for_current_device(&tw);
    if (rc != BPLG_OK) return rc;
    rc = ensure_smem_attr(li.func, li.smem);
    if (rc != BPLG_OK) return rc;
    int logn = ilog2(n);
    int spb = p.spb;
    if (p.io == 2) {
        int64_t ntiles = li.blocks;
        int slot_elems = fft_tma_slot_elems_layout(p.smem_layout, p.smem_pad, n, p.spb);
        int64_t grid = 0;
        rc = persistent_grid(li.func, li.threads, li.smem, ntiles, &grid);
        if (rc != BPLG_OK) return rc;
        void *args[] = {(void *)&in, (void *)&out, (void *)&tw, &logn, &spb, &batch, &ntiles, &slot_elems};
        cudaError_t e = cudaLaunchKernel(li.func, dim3(static_cast<unsigned>(grid)), dim3(li.threads), args,
                                         static_cast<size_t>(li.smem), s);
        return e == cudaSuccess ? BPLG_OK : launch_error(e, "fft pipelined launch", li.func, grid, li.threads, li.smem);
    }
    void *args[] = {(void *)&in, (void *)&out, (void *)&tw, &logn, &spb, &batch};
    cudaError_t e = cudaLaunchKernel(li.func, dim3(static_cast<unsigned>(li.blocks)), dim3(li.threads), args,
                                     static_cast<size_t>(li.smem), s);
    return e == cudaSuccess ? BPLG_OK : cuda_error(e, "fft launch");
}

}  // namespace bplg

namespace bplg {

// Read (and optionally clear) the device error word of this file's kernels
// on the current device.
int fft_device_status(int *flag, bool reset) {
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

// ---------------------------------------------------------------------------
// FFT entry point that allocates nothing.
//
// The regular entry point allocates its twiddle table with cudaMalloc the
// first time it runs on a device.  Some callers cannot allow that: code that
// runs under an allocator which owns all of the device's memory (a framework's
// caching allocator, a fixed real-time memory budget), code that must not
// trigger the implicit device synchronisation an allocation can cause, and
// code whose allocations are only permitted during start-up.  For them the
// twiddle table lives in the file-scope device array below, sized for
// transforms of at most kNoAllocMaxN points (64 KB): every GPU that loads the
// library holds it until the process exits.  The caller still provides the
// input and output buffers.
namespace bplg {

constexpr int kNoAllocMaxLog = 12;
constexpr int kNoAllocMaxN = 1 << kNoAllocMaxLog;
constexpr int kNoAllocMaxDevices = 64;

}  // namespace bplg

// W_M^k at [M + k] for M = 2 .. kNoAllocMaxN, as in the regular table.  The
// values are part of the module image (a static initializer written at build
// time from float64 values rounded once to float32), so the array is ready
// as soon as the module is loaded on a device: no fill kernel, no wait, and a
// module reloaded after cudaDeviceReset holds them again.
static __device__ __align__(256) float2 g_noalloc_twiddles[2 * bplg::kNoAllocMaxN] = {
#include "noalloc_twiddles.inc"
};

namespace bplg {
namespace {

std::mutex g_noalloc_mu;
const float2 *g_noalloc_addr[kNoAllocMaxDevices];  // device address of the array, per device

// Set-up, once per device, with that device current: look up the array's
// device address (in host code its name is only a stand-in for it, which a
// kernel must never be given).  Nothing is launched or waited for.
int noalloc_setup(const float2 **tw) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= kNoAllocMaxDevices) return set_error(BPLG_ERR_INVALID_ARG, "device index too large");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        float2 *ptr = nullptr;
        e = cudaGetSymbolAddress(reinterpret_cast<void **>(&ptr), g_noalloc_twiddles);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(no-alloc twiddles)");
        g_noalloc_addr[dev] = ptr;
    }
    *tw = g_noalloc_addr[dev];
    return BPLG_OK;
}

}  // namespace
}  // namespace bplg

using namespace bplg;

extern "C" int bplg_fft_batched_noalloc(const void *in, void *out, int64_t n, int64_t batch, int32_t dir,
                                        const bplg_plan *plan, void *stream) {
    clear_error();
    if (!in || !out) return set_error(BPLG_ERR_INVALID_ARG, "fft no-alloc: null buffer");
    if (n < 1 || batch < 1) return set_error(BPLG_ERR_INVALID_ARG, "fft no-alloc: n and batch must be >= 1");
    if (dir != -1 && dir != 1) return set_error(BPLG_ERR_INVALID_ARG, "fft no-alloc: dir must be -1 or +1");
    if (!is_pow2(n) || n < 2)
        return set_error(BPLG_ERR_UNSUPPORTED_SIZE, "fft no-alloc: n must be a power of two >= 2");
    if (n > kNoAllocMaxN)
        return set_error(BPLG_ERR_UNSUPPORTED_SIZE,
                         "fft no-alloc: n is above 4096, the size its static twiddle table holds; "
                         "use bplg_fft_batched for larger transforms");
    if (!aligned16(in) || !aligned16(out)) return set_error(BPLG_ERR_INVALID_ARG, "fft no-alloc: buffers must be 16-byte aligned");
    // the plan: the caller's, or a fixed default computed without any lookup
    bplg_plan p;
    if (plan) {
        p = *plan;
    } else {
        std::memset(&p, 0, sizeof(p));
        p.op = BPLG_OP_FFT;
        p.n = static_cast<int32_t>(n);
        p.P = p.radix = n >= 16 ? 16 : static_cast<int32_t>(n);
        const int64_t T = n / p.P;
        p.spb = static_cast<int32_t>(T >= 128 ? 1 : 128 / T);
        p.L = static_cast<int32_t>(p.spb * T);
        p.smem_pad = 1;
        p.io = T >= 32 ? 0 : 1;
    }
    if (p.op != BPLG_OP_FFT || !plan_structurally_valid(p, BPLG_F32, n, nullptr) || p.io > 1)
        return set_error(BPLG_ERR_INVALID_PLAN, "fft no-alloc: invalid plan (the pipelined io mode is not offered here)");
    const void *func = fft_func(p.radix, dir, p.smem_layout, p.smem_pad, p.io, p.L, ilog2(n));
    if (!func) return set_error(BPLG_ERR_INVALID_PLAN, "fft no-alloc: plan has no kernel");
    const int smem = fft_smem_bytes(p.radix, p.smem_layout, p.smem_pad, p.io, n, p.spb);
    const int64_t blocks = batch / p.spb + (batch % p.spb != 0 ? 1 : 0);
    int rc = check_grid(blocks, "fft no-alloc");
    if (rc != BPLG_OK) return rc;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaDeviceGetAttribute");
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, func);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncGetAttributes");
    if (p.L > fa.maxThreadsPerBlock) return set_error(BPLG_ERR_INVALID_PLAN, "fft no-alloc: block too large for the kernel");
    if (static_cast<int64_t>(smem) + static_cast<int64_t>(fa.sharedSizeBytes) > optin)
        return set_error(BPLG_ERR_INVALID_PLAN, "fft no-alloc: the plan's shared memory is above the per-block limit");
    if (smem > fa.maxDynamicSharedSizeBytes) {
        e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(max dynamic smem)");
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float2 *tw = nullptr;
    rc = noalloc_setup(&tw);
    if (rc != BPLG_OK) return rc;
    int logn = ilog2(n);
    int spb = p.spb;
    void *args[] = {(void *)&in, (void *)&out, (void *)&tw, &logn, &spb, &batch};
    e = cudaLaunchKernel(func, dim3(static_cast<unsigned>(blocks)), dim3(p.L), args, static_cast<size_t>(smem), s);
    return e == cudaSuccess ? BPLG_OK : cuda_error(e, "fft no-alloc launch");
}
