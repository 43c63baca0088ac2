// FFT of more than 2^14 points: two kernels (the multi-kernel transform of
// Section V-C, for signals too large for one block's shared memory).
//
// The signal of n = N1 N2 points is read as an N1 x N2 row-major matrix
// x[n1][n2] = x[n1 N2 + n2].  With n1 and k1 indexing N1, n2 and k2
// indexing N2 (W_M = exp(dir 2 pi i / M)):
//     X[k1 + N1 k2] = sum_n2 W_N2^(n2 k2) W_n^(n2 k1) sum_n1 W_N1^(n1 k1) x[n1][n2]
//   kernel 1 (columns): y[k1][n2] = W_n^(k1 n2) sum_n1 W_N1^(n1 k1) x[n1][n2];
//   kernel 2 (rows):    X[k1 + N1 k2] = sum_n2 W_N2^(n2 k2) y[k1][n2].
// Both inner transforms are the radix-16 Stockham stages of the
// size-specialised single-block kernel (compile-time schedule, padded
// exchanges in shared memory).
//
//   Kernel 1 takes spb adjacent columns of one signal per block: thread
//   (j, c) = (tid / spb, tid % spb), so a warp's loads of one row are spb
//   contiguous complex values; column c is exchanged in its own padded
//   buffer (stride skewed by one element so the columns fall in different
//   banks), and output k1 of column n2 is multiplied by W_n^(k1 n2) and
//   stored to y[k1][n2], again spb contiguous values per row.
//   Kernel 2 takes row_spb adjacent rows per block: loads are contiguous
//   within a row; the outputs are collected in shared memory and written
//   transposed, X[k1 + N1 k2] for row_spb consecutive k1 at a time.
//
// y lives in a scratch buffer owned by the library (allocated on first use
// per device and stream, grown to the largest n x batch seen), so in may
// equal out.
// W_n^m for n up to 2^24 is a product of two float64-generated tables:
// W_n^(m mod 4096) (one 4096-entry table per n, cached per device) and
// W_(n/4096)^(m div 4096) from the main twiddle table.
#include <algorithm>
#include <cstring>
#include <map>
#include <tuple>
#include <mutex>

#include "device_util.cuh"
#include "fft_common.cuh"
#include "internal.h"

namespace bplg {

int twiddles_for_current_device(const void **tw);

namespace {

constexpr int kLargeMinPassLog = 6;   // each inner transform has 2^6 .. 2^14 points
constexpr int kLargeMaxPassLog = 14;
constexpr int kFineLog = 12;          // fine twiddle table: W_n^j, j < 4096

__device__ __forceinline__ float2 twiddle_n(const float2 *__restrict__ tw, const float2 *__restrict__ fine, int logn,
                                            uint32_t m, int dir) {
    const float2 lo = __ldg(fine + (m & ((1u << kFineLog) - 1)));
    const float2 hi = __ldg(tw + (1u << (logn - kFineLog)) + (m >> kFineLog));
    float2 w = cmul(lo, hi);
    if (dir > 0) w.y = -w.y;
    return w;
}

__host__ __device__ constexpr int col_stride(int n1) { return n1 + n1 / 16 + 1; }  // float2, skewed
// rows of the row kernel: a pad of 16 / R float2 (R = rows per block <= 16)
// puts the R rows of the transposed read-out 32 / R banks apart, so the 16
// lanes of each half-warp (16 / R columns x R rows) hit 16 bank pairs
__host__ __device__ constexpr int row_stride(int n2, int log_rows) {
    return n2 + n2 / 16 + (log_rows <= 4 ? (16 >> log_rows) : 1);
}

template <int LOGN1, int DIR>
__global__ void __launch_bounds__(1024)
    fft_col_kernel(const float2 *in, float2 *y, const float2 *__restrict__ tw, const float2 *__restrict__ fine,
                   int logn, int log_cols) {
    using S = FftShape<16, LOGN1>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *cols = reinterpret_cast<float2 *>(smem_raw);
    const int logn2 = logn - LOGN1;
    const int64_t N = int64_t(1) << logn;
    const int64_t N2 = int64_t(1) << logn2;
    const int tid = threadIdx.x;
    const int c = tid & ((1 << log_cols) - 1);
    const int j = tid >> log_cols;
    const int64_t tiles = N2 >> log_cols;  // column tiles per signal
    const int64_t sig = blockIdx.x / tiles;
    const int64_t n2 = ((blockIdx.x - sig * tiles) << log_cols) + c;
    const float2 *g = in + sig * N + n2;
    float2 v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = __ldcs(g + static_cast<int64_t>(j + m * S::T) * N2);
    float2 *yo = y + sig * N + n2;
    auto store = [&](int k1, float2 val) {
        const float2 w = twiddle_n(tw, fine, logn, static_cast<uint32_t>(k1) * static_cast<uint32_t>(n2), DIR);
        __stcs(yo + static_cast<int64_t>(k1) * N2, cmul(val, w));
    };
    fft_fixed_stages_st<16, LOGN1, DIR, 0, 0>(v, cols + c * col_stride(1 << LOGN1), nullptr, j, tw, store);
}

template <int LOGN2, int DIR>
__global__ void __launch_bounds__(1024)
    fft_row_kernel(const float2 *y, float2 *out, const float2 *__restrict__ tw, int logn, int log_rows) {
    using S = FftShape<16, LOGN2>;
    constexpr int N2 = 1 << LOGN2;
    const int RS = row_stride(N2, log_rows);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *rows = reinterpret_cast<float2 *>(smem_raw);
    const int logn1 = logn - LOGN2;
    const int64_t N = int64_t(1) << logn;
    const int64_t N1 = int64_t(1) << logn1;
    const int R = 1 << log_rows;
    const int tid = threadIdx.x;
    const int rr = tid >> S::LOGT;
    const int j = tid & (S::T - 1);
    const int64_t tiles = N1 >> log_rows;  // row tiles per signal
    const int64_t sig = blockIdx.x / tiles;
    const int64_t k1_0 = (blockIdx.x - sig * tiles) << log_rows;
    const float2 *g = y + sig * N + (k1_0 + rr) * N2 + j;
    float2 v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = __ldcs(g + m * S::T);
    float2 *row = rows + rr * RS;
    auto store = [&](int k2, float2 val) { row[pad_g<16>(k2)] = val; };
    fft_fixed_stages_st<16, LOGN2, DIR, 0, 0, true>(v, row, nullptr, j, tw, store);
    __syncthreads();
    // transposed write-out: R consecutive k1 per output column k2
    float2 *o = out + sig * N + k1_0;
    for (int e = tid; e < R * N2; e += blockDim.x) {
        const int r2 = e & (R - 1);
        const int k2 = e >> log_rows;
        __stcs(o + r2 + N1 * k2, rows[r2 * RS + pad_g<16>(k2)]);
    }
}

template <int DIR>
const void *col_func(int l1) {
    switch (l1) {
        case 6: return reinterpret_cast<const void *>(&fft_col_kernel<6, DIR>);
        case 7: return reinterpret_cast<const void *>(&fft_col_kernel<7, DIR>);
        case 8: return reinterpret_cast<const void *>(&fft_col_kernel<8, DIR>);
        case 9: return reinterpret_cast<const void *>(&fft_col_kernel<9, DIR>);
        case 10: return reinterpret_cast<const void *>(&fft_col_kernel<10, DIR>);
        case 11: return reinterpret_cast<const void *>(&fft_col_kernel<11, DIR>);
        case 12: return reinterpret_cast<const void *>(&fft_col_kernel<12, DIR>);
        case 13: return reinterpret_cast<const void *>(&fft_col_kernel<13, DIR>);
        case 14: return reinterpret_cast<const void *>(&fft_col_kernel<14, DIR>);
        default: return nullptr;
    }
}

template <int DIR>
const void *row_func(int l2) {
    switch (l2) {
        case 6: return reinterpret_cast<const void *>(&fft_row_kernel<6, DIR>);
        case 7: return reinterpret_cast<const void *>(&fft_row_kernel<7, DIR>);
        case 8: return reinterpret_cast<const void *>(&fft_row_kernel<8, DIR>);
        case 9: return reinterpret_cast<const void *>(&fft_row_kernel<9, DIR>);
        case 10: return reinterpret_cast<const void *>(&fft_row_kernel<10, DIR>);
        case 11: return reinterpret_cast<const void *>(&fft_row_kernel<11, DIR>);
        case 12: return reinterpret_cast<const void *>(&fft_row_kernel<12, DIR>);
        case 13: return reinterpret_cast<const void *>(&fft_row_kernel<13, DIR>);
        case 14: return reinterpret_cast<const void *>(&fft_row_kernel<14, DIR>);
        default: return nullptr;
    }
}

// fine twiddles W_n^j (j < 4096) in float64, rounded once
__global__ void fine_twiddle_kernel(float2 *t, int logn) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= (1 << kFineLog)) return;
    double sn, cs;
    sincospi(-2.0 * static_cast<double>(j) / static_cast<double>(int64_t(1) << logn), &sn, &cs);
    t[j] = make_float2(static_cast<float>(cs), static_cast<float>(sn));
}

std::mutex g_mu;
std::map<std::pair<int, int>, float2 *> g_fine;       // (device, log n)
// (device, stream, tag) -> (buffer, bytes)
std::map<std::tuple<int, cudaStream_t, int>, std::pair<void *, size_t>> g_scratch;

int fine_twiddles(int logn, const float2 **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_fine.find({dev, logn});
    if (it != g_fine.end()) {
        *out = it->second;
        return BPLG_OK;
    }
    float2 *p = nullptr;
    e = cudaMalloc(&p, sizeof(float2) << kFineLog);
    if (e != cudaSuccess) return cuda_error(e, "fine twiddle cudaMalloc");
    cudaStream_t st;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaFree(p);
        return cuda_error(e, "fine twiddle stream");
    }
    fine_twiddle_kernel<<<(1 << kFineLog) / 256, 256, 0, st>>>(p, logn);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (e != cudaSuccess) {
        cudaFree(p);
        return cuda_error(e, "fine twiddle generation");
    }
    g_fine[{dev, logn}] = p;
    *out = p;
    return BPLG_OK;
}

}  // namespace

// Library-owned scratch per (device, stream, tag): launches on one stream
// are ordered, so they may share it, and concurrent streams get their own.
// It grows, never shrinks; a growth first waits for the stream (earlier
// launches on it may still use the old buffer), so calls that need no growth
// never synchronise.
int stream_scratch(int tag, size_t bytes, cudaStream_t s, void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lock(g_mu);
    auto &slot = g_scratch[std::make_tuple(dev, s, tag)];
    if (slot.second < bytes) {
        if (slot.first) {
            e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_error(e, "scratch growth");
            cudaFree(slot.first);
            slot = {nullptr, 0};
        }
        void *p = nullptr;
        e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) return cuda_error(e, "fft scratch cudaMalloc");
        slot = {p, bytes};
    }
    *out = slot.first;
    return BPLG_OK;
}

namespace {

bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

}  // namespace

int fft_large_smem_bytes(const bplg_plan &p, int64_t n, int pass) {
    const int l1 = p.n1_log, l2 = ilog2(n) - p.n1_log;
    if (pass == 0) return p.spb * col_stride(1 << l1) * 8;
    return p.row_spb * row_stride(1 << l2, ilog2(p.row_spb)) * 8;
}

bool fft_large_plan_valid(const bplg_plan &p, int64_t n, std::string *why) {
    auto fail = [&](const char *m) {
        if (why) *why = m;
        return false;
    };
    const int logn = ilog2(n);
    const int l1 = p.n1_log, l2 = logn - p.n1_log;
    if (p.P != 16 || p.radix != 16) return fail("FFT above 16384 points: radix and P are 16");
    if (l1 < kLargeMinPassLog || l1 > kLargeMaxPassLog || l2 < kLargeMinPassLog || l2 > kLargeMaxPassLog)
        return fail("FFT above 16384 points: both N1 = 2^n1_log and n / N1 between 64 and 16384");
    if (!pow2_in(p.spb, 1, 64) || !pow2_in(p.row_spb, 1, 64)) return fail("FFT above 16384 points: spb, row_spb in 1..64");
    if (fft_large_smem_bytes(p, n, 0) > 227 * 1024 || fft_large_smem_bytes(p, n, 1) > 227 * 1024)
        return fail("FFT above 16384 points: shared memory above 227 KB per block");
    const int64_t t1 = int64_t(p.spb) << (l1 - 4), t2 = int64_t(p.row_spb) << (l2 - 4);
    if (t1 < 32 || t1 > 1024 || t2 < 32 || t2 > 1024)
        return fail("FFT above 16384 points: 32 to 1024 threads per block in both kernels");
    if (p.L != t1) return fail("FFT above 16384 points: L = spb * N1 / 16");
    if (p.smem_pad != 1 || p.smem_layout != 0 || p.io != 0 || p.shuffle != 0 || p.pattern != 0 || p.cr_switch != 0 ||
        p.reserved != 0)
        return fail("FFT above 16384 points: padded interleaved exchanges, io 0, other knobs 0");
    return true;
}

void fft_large_finalize(bplg_plan *p, int64_t n) {
    p->n = static_cast<int32_t>(n);
    p->P = p->radix = 16;
    p->L = p->n1_log >= 4 ? (p->spb << (p->n1_log - 4)) : 0;
    p->smem_pad = 1;
    p->smem_layout = p->io = p->shuffle = p->pattern = p->cr_switch = p->reserved = 0;
    p->S = static_cast<int32_t>(std::max(fft_large_smem_bytes(*p, n, 0), fft_large_smem_bytes(*p, n, 1)) / 8);
}

std::vector<bplg_plan> fft_large_enumerate(int64_t n) {
    std::vector<bplg_plan> out;
    const int logn = ilog2(n);
    for (int l1 = kLargeMinPassLog; l1 <= kLargeMaxPassLog; ++l1) {
        for (int c = 1; c <= 64; c *= 2) {
            for (int r = 1; r <= 64; r *= 2) {
                bplg_plan p;
                std::memset(&p, 0, sizeof(p));
                p.op = BPLG_OP_FFT;
                p.n1_log = l1;
                p.spb = c;
                p.row_spb = r;
                fft_large_finalize(&p, n);
                if (fft_large_plan_valid(p, n, nullptr) && logn - l1 >= kLargeMinPassLog) out.push_back(p);
            }
        }
    }
    return out;
}

bool fft_large_launch_info(const bplg_plan &p, int64_t n, int64_t batch, int dir, int pass, Launch *out) {
    if (!fft_large_plan_valid(p, n, nullptr)) return false;
    const int l1 = p.n1_log, l2 = ilog2(n) - p.n1_log;
    if (pass == 0) {
        out->func = dir < 0 ? col_func<-1>(l1) : col_func<1>(l1);
        out->threads = p.spb << (l1 - 4);
        out->blocks = batch * ((int64_t(1) << l2) / p.spb);
    } else {
        out->func = dir < 0 ? row_func<-1>(l2) : row_func<1>(l2);
        out->threads = p.row_spb << (l2 - 4);
        out->blocks = batch * ((int64_t(1) << l1) / p.row_spb);
    }
    out->smem = fft_large_smem_bytes(p, n, pass);
    return out->func != nullptr;
}

int fft_large_launch(const bplg_plan &p, const void *in, void *out, int64_t n, int64_t batch, int dir,
                     cudaStream_t s) {
    Launch l0, l1;
    if (!fft_large_launch_info(p, n, batch, dir, 0, &l0) || !fft_large_launch_info(p, n, batch, dir, 1, &l1))
        return set_error(BPLG_ERR_INVALID_PLAN, "fft (two kernels): plan has no kernel");
    int rc = check_grid(l0.blocks > l1.blocks ? l0.blocks : l1.blocks, "fft (two kernels)");
    if (rc != BPLG_OK) return rc;
    const void *tw = nullptr;
    rc = twiddles_for_current_device(&tw);
    if (rc != BPLG_OK) return rc;
    int logn = ilog2(n);
    const float2 *fine = nullptr;
    rc = fine_twiddles(logn, &fine);
    if (rc != BPLG_OK) return rc;
    void *y = nullptr;
    rc = stream_scratch(kScratchLargeFft, static_cast<size_t>(n) * static_cast<size_t>(batch) * sizeof(float2), s, &y);
    if (rc != BPLG_OK) return rc;
    rc = ensure_smem_attr(l0.func, l0.smem);
    if (rc == BPLG_OK) rc = ensure_smem_attr(l1.func, l1.smem);
    if (rc != BPLG_OK) return rc;
    int log_cols = ilog2(p.spb), log_rows = ilog2(p.row_spb);
    const float2 *x = static_cast<const float2 *>(in);
    float2 *yy = static_cast<float2 *>(y);
    float2 *o = static_cast<float2 *>(out);
    void *a0[] = {(void *)&x, (void *)&yy, (void *)&tw, (void *)&fine, &logn, &log_cols};
    cudaError_t e = cudaLaunchKernel(l0.func, dim3(static_cast<unsigned>(l0.blocks)), dim3(l0.threads), a0,
                                     static_cast<size_t>(l0.smem), s);
    if (e != cudaSuccess) return launch_error(e, "fft column kernel", l0.func, l0.blocks, l0.threads, l0.smem);
    const float2 *yc = yy;
    void *a1[] = {(void *)&yc, (void *)&o, (void *)&tw, &logn, &log_rows};
    e = cudaLaunchKernel(l1.func, dim3(static_cast<unsigned>(l1.blocks)), dim3(l1.threads), a1,
                         static_cast<size_t>(l1.smem), s);
    return e == cudaSuccess ? BPLG_OK : launch_error(e, "fft row kernel", l1.func, l1.blocks, l1.threads, l1.smem);
}

}  // namespace bplg
