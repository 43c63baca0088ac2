// Uneven-size batches in one launch: problems of different sizes and kinds
// (the uniform batches of G problems of Section IV-A generalised to mixed
// sizes) are grouped by (operation, size) into units, largest first, and
// three persistent kernels -- scan, Stockham FFT, register-level CR/PCR --
// pull units from one atomic counter each until the work runs out.  The
// counter reset and the three kernels (on forked branches) are captured once
// into a CUDA graph, so every run is a single graph launch.
//
// Units hold up to spb problems of one size; within a unit the layout is
// the batched kernels' (one signal per T threads), but every problem has its
// own input and output pointers, so problems need not be contiguous.
//   scan     256 threads; P = 16 for n <= 4096, else 32 (T <= 256): enough
//            bytes in flight per thread to cover the memory latency
//   FFT      512 threads, two blocks per SM; radix 16 (mixed-radix first
//            stage), T = n / 16, every size with the compile-time stage
//            schedule (one non-inlined function per size)
//   tridiag  512 threads, two blocks per SM; P = 16; the Wang-Mou divide and
//            conquer (each thread's 16 equations by a Thomas sweep, then
//            radix-2 merges)
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "device_util.cuh"
#include "fft_common.cuh"
#include "internal.h"
#include "tridiag_common.cuh"
#include "tridiag_wm.cuh"

namespace bplg {

struct ItemDesc {
    const void *in0, *in1, *in2, *in3;
    void *out;
};

struct UnitDesc {
    int32_t first;  // first item of the unit (items of a unit are consecutive)
    int32_t count;  // problems in the unit
    int32_t logn;
    int32_t flags;  // scan: dtype; FFT: direction
};

constexpr int kUnevenScanThreads = 256;
constexpr int kUnevenFftThreads = 512;
constexpr int kUnevenTriThreads = 512;
constexpr int kUnevenMinLog = 5;
constexpr int kUnevenMaxLog = 13;

__host__ __device__ inline int uneven_scan_P(int logn) { return logn <= 12 ? 16 : 32; }

// ------------------------------------------------------------------ scan
template <typename E, int P>
__device__ __forceinline__ void scan_unit(const ItemDesc *items, const UnitDesc &U, E *warp_tot) {
    const int logT = U.logn - clog2(P);
    const int T = 1 << logT;
    const int tid = threadIdx.x;
    const int s = tid >> logT;
    const int t = tid & (T - 1);
    const bool active = s < U.count;
    const E *in = nullptr;
    E *out = nullptr;
    if (active) {
        in = static_cast<const E *>(items[U.first + s].in0) + t * P;
        out = static_cast<E *>(items[U.first + s].out) + t * P;
    }
    E v[P];
    if (active) {
        load_run<E, P>(in, v);
    } else {
#pragma unroll
        for (int i = 0; i < P; ++i) v[i] = E(0);
    }
#pragma unroll
    for (int i = 1; i < P; ++i) v[i] += v[i - 1];
    const int lane = tid & 31;
    const int width = T < 32 ? T : 32;
    const int lane_in_seg = lane & (width - 1);
    E incl = seg_scan<0>(v[P - 1], lane_in_seg, width);
    E excl = __shfl_up_sync(kFullMask, incl, 1, width);
    if (lane_in_seg == 0) excl = E(0);
    if (T > 32) {
        const int warp = tid >> 5;
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        const int wps = T >> 5;
        const int wl = warp & (wps - 1);
        E w = (lane < wps) ? warp_tot[(warp - wl) + lane] : E(0);
        w = seg_scan<0>(w, lane, 32);
        E woff = __shfl_sync(kFullMask, w, wl > 0 ? wl - 1 : 0);
        if (wl == 0) woff = E(0);
        excl += woff;
    }
#pragma unroll
    for (int i = 0; i < P; ++i) v[i] += excl;
    if (active) store_run<E, P>(out, v);
}

template <typename E>
__device__ __forceinline__ void scan_unit_dispatch(const ItemDesc *items, const UnitDesc &U, E *warp_tot) {
    switch (uneven_scan_P(U.logn)) {
        case 4: scan_unit<E, 4>(items, U, warp_tot); break;
        case 8: scan_unit<E, 8>(items, U, warp_tot); break;
        case 16: scan_unit<E, 16>(items, U, warp_tot); break;
        default: scan_unit<E, 32>(items, U, warp_tot); break;
    }
}

__global__ void __launch_bounds__(kUnevenScanThreads)
    uneven_scan_kernel(const ItemDesc *items, const UnitDesc *units, int nunits, int *counter) {
    __shared__ int s_unit;
    __shared__ int32_t tot_i[32];
    __shared__ float tot_f[32];
    if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1);
    __syncthreads();
    for (;;) {
        const int u = s_unit;
        if (u >= nunits) break;
        int next = 0;
        if (threadIdx.x == 0) next = atomicAdd(counter, 1);  // the next unit, fetched while this one runs
        const UnitDesc U = units[u];
        if (U.flags == BPLG_I32)
            scan_unit_dispatch<int32_t>(items, U, tot_i);
        else
            scan_unit_dispatch<float>(items, U, tot_f);
        __syncthreads();  // warp totals are reused by the next unit; every thread has read s_unit
        if (threadIdx.x == 0) s_unit = next;
        __syncthreads();
    }
}

// ------------------------------------------------------------------- FFT
// One FFT unit: the compile-time stage schedule of the size-specialised
// batched kernel (constant exchange offsets, unrolled stages).  Not inlined:
// each size keeps its own register allocation instead of all of them
// merging into the kernel's.
template <int LOGN, int DIR>
__device__ __noinline__ void fft_unit_fixed(const ItemDesc *items, const UnitDesc &U,
                                               const float2 *__restrict__ tw, float2 *buf) {
    using S = FftShape<16, LOGN>;
    const int tid = threadIdx.x;
    const int s = tid >> S::LOGT;
    const int j = tid & (S::T - 1);
    const bool active = s < U.count;
    float2 *b2 = buf + s * sig_stride<0, 1>(1 << LOGN);
    const float2 *in = active ? static_cast<const float2 *>(items[U.first + s].in0) + j : nullptr;
    float2 *out = active ? static_cast<float2 *>(items[U.first + s].out) : nullptr;
    float2 v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = active ? __ldcs(in + m * S::T) : make_float2(0.f, 0.f);
    fft_fixed_stages<16, LOGN, DIR, 0, 0>(v, b2, nullptr, j, tw, out, active);
}

template <int DIR>
__device__ __forceinline__ void fft_unit_any(const ItemDesc *items, const UnitDesc &U, const float2 *__restrict__ tw,
                                             float2 *buf) {
    switch (U.logn) {
        case 5: fft_unit_fixed<5, DIR>(items, U, tw, buf); break;
        case 6: fft_unit_fixed<6, DIR>(items, U, tw, buf); break;
        case 7: fft_unit_fixed<7, DIR>(items, U, tw, buf); break;
        case 8: fft_unit_fixed<8, DIR>(items, U, tw, buf); break;
        case 9: fft_unit_fixed<9, DIR>(items, U, tw, buf); break;
        case 10: fft_unit_fixed<10, DIR>(items, U, tw, buf); break;
        case 11: fft_unit_fixed<11, DIR>(items, U, tw, buf); break;
        case 12: fft_unit_fixed<12, DIR>(items, U, tw, buf); break;
        case 13: fft_unit_fixed<13, DIR>(items, U, tw, buf); break;
        default: break;  // sizes are checked on the host: 2^5 .. 2^13
    }
}

__global__ void __launch_bounds__(kUnevenFftThreads, 2)
    uneven_fft_kernel(const ItemDesc *items, const UnitDesc *units, int nunits, int *counter,
                      const float2 *__restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_unit;
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1);
    __syncthreads();
    for (;;) {
        const int u = s_unit;
        if (u >= nunits) break;
        int next = 0;
        if (threadIdx.x == 0) next = atomicAdd(counter, 1);  // the next unit, fetched while this one runs
        const UnitDesc U = units[u];
        if (U.flags < 0)
            fft_unit_any<-1>(items, U, tw, buf);
        else
            fft_unit_any<1>(items, U, tw, buf);
        __syncthreads();  // the exchange buffer is reused by the next unit; every thread has read s_unit
        if (threadIdx.x == 0) s_unit = next;
        __syncthreads();
    }
}

// --------------------------------------------------------------- tridiag
// A unit of systems of one size solved with the Wang-Mou divide and conquer
// (radix-2 merges, shuffles inside a warp, shared memory across warps).
// (Feeding the next unit through a shared-memory slot while one is solved
// was measured slower, with per-thread asynchronous copies and with bulk
// copies alike: 76 and 90 us against 53 us for the 4096-system batch.)
constexpr int kUnevenTriP = 16;

template <int P>
__device__ __forceinline__ void tri_unit(const ItemDesc *items, const UnitDesc &U, float4 *smem) {
    const int log_tps = U.logn - clog2(P);
    const int s = threadIdx.x >> log_tps;
    const int t = threadIdx.x & ((1 << log_tps) - 1);
    const bool active = s < U.count;
    const float *ga = nullptr, *gb = nullptr, *gc = nullptr, *gd = nullptr;
    float *x = nullptr;
    if (active) {
        const ItemDesc &it = items[U.first + s];
        const int off = t * P;
        ga = static_cast<const float *>(it.in0) + off;
        gb = static_cast<const float *>(it.in1) + off;
        gc = static_cast<const float *>(it.in2) + off;
        gd = static_cast<const float *>(it.in3) + off;
        x = static_cast<float *>(it.out) + off;
    }
    wm::wm_solve<P, 2, 1>(ga, gb, gc, gd, x, active, log_tps, smem);
}

__global__ void __launch_bounds__(kUnevenTriThreads, 2)
    uneven_tri_kernel(const ItemDesc *items, const UnitDesc *units, int nunits, int *counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_unit;
    float4 *smem = reinterpret_cast<float4 *>(smem_raw);
    if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1);
    __syncthreads();
    for (;;) {
        const int u = s_unit;
        if (u >= nunits) break;
        int next = 0;
        if (threadIdx.x == 0) next = atomicAdd(counter, 1);  // the next unit, fetched while this one runs
        const UnitDesc U = units[u];
        tri_unit<kUnevenTriP>(items, U, smem);
        __syncthreads();  // the exchange buffers are reused by the next unit; every thread has read s_unit
        if (threadIdx.x == 0) s_unit = next;
        __syncthreads();
    }
}

// ------------------------------------------------------------------ host
namespace {

int fft_uneven_smem() {
    // largest padded tile over n = 32 .. 8192 with 512 threads of radix 16
    int best = 0;
    for (int l = kUnevenMinLog; l <= kUnevenMaxLog; ++l) {
        const int n = 1 << l;
        const int spb = kUnevenFftThreads / (n / 16);
        best = std::max(best, spb * sig_stride<0, 1>(n) * 8);
    }
    return best;
}

int tri_uneven_smem() {
    // the Wang-Mou exchanges: two parities x (first, last) x one float4 per thread
    return 4 * 16 * kUnevenTriThreads;
}

int units_per(int op, int logn) {
    if (op == BPLG_OP_SCAN) return kUnevenScanThreads / ((1 << logn) / uneven_scan_P(logn));
    if (op == BPLG_OP_FFT) return kUnevenFftThreads / ((1 << logn) / 16);
    return kUnevenTriThreads / ((1 << logn) / kUnevenTriP);
}

}  // namespace

struct UnevenBatch {
    int device = 0;
    ItemDesc *d_items = nullptr;
    UnitDesc *d_units = nullptr;
    int *d_counters = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t nitems = 0;
    int nunits[3] = {0, 0, 0};
    ~UnevenBatch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (d_items) cudaFree(d_items);
        if (d_units) cudaFree(d_units);
        if (d_counters) cudaFree(d_counters);
    }
};

int uneven_create(const bplg_item *items, int64_t count, UnevenBatch **out) {
    if (!items || count < 1 || count > (int64_t(1) << 30) || !out)
        return set_error(BPLG_ERR_INVALID_ARG, "uneven: bad arguments");
    // validate and sort: per op, by size descending (largest units first)
    struct Key {
        int op, logn, flags;
        int64_t idx;
    };
    std::vector<Key> keys;
    keys.reserve(static_cast<size_t>(count));
    for (int64_t i = 0; i < count; ++i) {
        const bplg_item &it = items[i];
        if (it.op != BPLG_OP_SCAN && it.op != BPLG_OP_FFT && it.op != BPLG_OP_TRIDIAG)
            return set_error(BPLG_ERR_INVALID_ARG, "uneven: item op must be SCAN, FFT or TRIDIAG");
        if (!is_pow2(it.n) || it.n < (1 << kUnevenMinLog) || it.n > (1 << kUnevenMaxLog))
            return set_error(BPLG_ERR_UNSUPPORTED_SIZE, "uneven: item n must be a power of two in [32, 8192]");
        const int nin = it.op == BPLG_OP_TRIDIAG ? 4 : 1;
        for (int k = 0; k < nin; ++k)
            if (!it.in[k] || !aligned16(it.in[k])) return set_error(BPLG_ERR_INVALID_ARG, "uneven: null or misaligned input");
        if (!it.out || !aligned16(it.out)) return set_error(BPLG_ERR_INVALID_ARG, "uneven: null or misaligned output");
        int flags = 0;
        if (it.op == BPLG_OP_SCAN) {
            if (it.dtype != BPLG_I32 && it.dtype != BPLG_F32) return set_error(BPLG_ERR_INVALID_ARG, "uneven: scan dtype");
            flags = it.dtype;
        } else if (it.op == BPLG_OP_FFT) {
            if (it.dir != -1 && it.dir != 1) return set_error(BPLG_ERR_INVALID_ARG, "uneven: FFT dir must be -1 or +1");
            flags = it.dir;
        }
        keys.push_back(Key{it.op, ilog2(it.n), flags, i});
    }
    std::stable_sort(keys.begin(), keys.end(), [](const Key &x, const Key &y) {
        if (x.op != y.op) return x.op < y.op;
        if (x.logn != y.logn) return x.logn > y.logn;
        return x.flags < y.flags;
    });
    std::vector<ItemDesc> h_items(keys.size());
    std::vector<UnitDesc> h_units;
    int unit_off[3] = {0, 0, 0};
    for (size_t k = 0; k < keys.size(); ++k) {
        const bplg_item &it = items[keys[k].idx];
        h_items[k] = ItemDesc{it.in[0], it.in[1], it.in[2], it.in[3], it.out};
    }
    auto opslot = [](int op) { return op == BPLG_OP_SCAN ? 0 : (op == BPLG_OP_FFT ? 1 : 2); };
    std::unique_ptr<UnevenBatch> ub(new UnevenBatch());
    for (int slot = 0; slot < 3; ++slot) {
        unit_off[slot] = static_cast<int>(h_units.size());
        size_t k = 0;
        while (k < keys.size()) {
            if (opslot(keys[k].op) != slot) {
                ++k;
                continue;
            }
            const int cap = units_per(keys[k].op, keys[k].logn);
            size_t e = k;
            while (e < keys.size() && e - k < static_cast<size_t>(cap) && keys[e].op == keys[k].op &&
                   keys[e].logn == keys[k].logn && keys[e].flags == keys[k].flags)
                ++e;
            h_units.push_back(UnitDesc{static_cast<int32_t>(k), static_cast<int32_t>(e - k), keys[k].logn, keys[k].flags});
            k = e;
        }
        ub->nunits[slot] = static_cast<int>(h_units.size()) - unit_off[slot];
    }
    ub->nitems = count;
    cudaError_t e = cudaGetDevice(&ub->device);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    const void *tw = nullptr;
    int rc = twiddles_for_current_device(&tw);
    if (rc != BPLG_OK) return rc;
    if ((e = cudaMalloc(&ub->d_items, h_items.size() * sizeof(ItemDesc))) != cudaSuccess) return cuda_error(e, "uneven items");
    if ((e = cudaMalloc(&ub->d_units, std::max<size_t>(1, h_units.size()) * sizeof(UnitDesc))) != cudaSuccess)
        return cuda_error(e, "uneven units");
    if ((e = cudaMalloc(&ub->d_counters, 4 * sizeof(int))) != cudaSuccess) return cuda_error(e, "uneven counters");
    if ((e = cudaMemcpy(ub->d_items, h_items.data(), h_items.size() * sizeof(ItemDesc), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return cuda_error(e, "uneven upload");
    if (!h_units.empty() && (e = cudaMemcpy(ub->d_units, h_units.data(), h_units.size() * sizeof(UnitDesc),
                                            cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_error(e, "uneven upload");

    const int fsm = fft_uneven_smem(), tsm = tri_uneven_smem();
    rc = ensure_smem_attr(reinterpret_cast<const void *>(&uneven_fft_kernel), fsm);
    if (rc != BPLG_OK) return rc;
    rc = ensure_smem_attr(reinterpret_cast<const void *>(&uneven_tri_kernel), tsm);
    if (rc != BPLG_OK) return rc;
    int64_t g_scan = 0, g_fft = 0, g_tri = 0;
    rc = persistent_grid(reinterpret_cast<const void *>(&uneven_scan_kernel), kUnevenScanThreads, 0,
                         std::max(1, ub->nunits[0]), &g_scan);
    if (rc == BPLG_OK)
        rc = persistent_grid(reinterpret_cast<const void *>(&uneven_fft_kernel), kUnevenFftThreads, fsm,
                             std::max(1, ub->nunits[1]), &g_fft);
    if (rc == BPLG_OK)
        rc = persistent_grid(reinterpret_cast<const void *>(&uneven_tri_kernel), kUnevenTriThreads, tsm,
                             std::max(1, ub->nunits[2]), &g_tri);
    if (rc != BPLG_OK) return rc;

    // capture: counter reset, then the three kernels on forked branches
    cudaStream_t s0 = nullptr, s1 = nullptr, s2 = nullptr;
    cudaEvent_t fork = nullptr, j1 = nullptr, j2 = nullptr;
    auto cleanup = [&]() {
        if (fork) cudaEventDestroy(fork);
        if (j1) cudaEventDestroy(j1);
        if (j2) cudaEventDestroy(j2);
        if (s0) cudaStreamDestroy(s0);
        if (s1) cudaStreamDestroy(s1);
        if (s2) cudaStreamDestroy(s2);
    };
    if ((e = cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&s1, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&j1, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&j2, cudaEventDisableTiming)) != cudaSuccess) {
        cleanup();
        return cuda_error(e, "uneven capture set-up");
    }
    const ItemDesc *di = ub->d_items;
    const UnitDesc *du = ub->d_units;
    int *dc = ub->d_counters;
    e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(dc, 0, 4 * sizeof(int), s0);
        cudaEventRecord(fork, s0);
        cudaStreamWaitEvent(s1, fork, 0);
        cudaStreamWaitEvent(s2, fork, 0);
        if (ub->nunits[0] > 0)
            uneven_scan_kernel<<<static_cast<unsigned>(g_scan), kUnevenScanThreads, 0, s0>>>(
                di, du + unit_off[0], ub->nunits[0], dc + 0);
        if (ub->nunits[1] > 0)
            uneven_fft_kernel<<<static_cast<unsigned>(g_fft), kUnevenFftThreads, fsm, s1>>>(
                di, du + unit_off[1], ub->nunits[1], dc + 1, static_cast<const float2 *>(tw));
        if (ub->nunits[2] > 0)
            uneven_tri_kernel<<<static_cast<unsigned>(g_tri), kUnevenTriThreads, tsm, s2>>>(
                di, du + unit_off[2], ub->nunits[2], dc + 2);
        cudaEventRecord(j1, s1);
        cudaEventRecord(j2, s2);
        cudaStreamWaitEvent(s0, j1, 0);
        cudaStreamWaitEvent(s0, j2, 0);
        e = cudaStreamEndCapture(s0, &ub->graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ub->exec, ub->graph, 0);
    cleanup();
    if (e != cudaSuccess) return cuda_error(e, "uneven graph capture");
    *out = ub.release();
    return BPLG_OK;
}

int uneven_launch(UnevenBatch *ub, cudaStream_t s) {
    if (!ub) return set_error(BPLG_ERR_INVALID_ARG, "uneven: null handle");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev != ub->device) return set_error(BPLG_ERR_INVALID_ARG, "uneven: handle made on another device");
    e = cudaGraphLaunch(ub->exec, s);
    return e == cudaSuccess ? BPLG_OK : cuda_error(e, "uneven graph launch");
}

void uneven_destroy(UnevenBatch *ub) { delete ub; }


int uneven_counts(const UnevenBatch *ub, int32_t *units) {
    for (int k = 0; k < 3; ++k) units[k] = ub->nunits[k];
    return BPLG_OK;
}

}  // namespace bplg

using namespace bplg;

extern "C" {

int bplg_uneven_create(const bplg_item *items, int64_t count, bplg_uneven_handle *out) {
    clear_error();
    UnevenBatch *ub = nullptr;
    int rc = uneven_create(items, count, &ub);
    if (rc != BPLG_OK) return rc;
    *out = reinterpret_cast<bplg_uneven_handle>(ub);
    return BPLG_OK;
}

int bplg_uneven_launch(bplg_uneven_handle h, void *stream) {
    clear_error();
    return uneven_launch(reinterpret_cast<UnevenBatch *>(h), static_cast<cudaStream_t>(stream));
}

int bplg_uneven_units(bplg_uneven_handle h, int32_t *units_scan_fft_tridiag) {
    clear_error();
    if (!h || !units_scan_fft_tridiag) return set_error(BPLG_ERR_INVALID_ARG, "uneven: null argument");
    return uneven_counts(reinterpret_cast<const UnevenBatch *>(h), units_scan_fft_tridiag);
}

int bplg_uneven_destroy(bplg_uneven_handle h) {
    clear_error();
    uneven_destroy(reinterpret_cast<UnevenBatch *>(h));
    return BPLG_OK;
}

}  // extern "C"
