// FFT of a length n that is not a power of two, by Bluestein's chirp
// identity over the library's power-of-two Stockham FFTs.  (The paper keeps
// to N = r^n; this extends the FFT entry point to every length.)
//
// With jk = (j^2 + k^2 - (k - j)^2) / 2 the DFT factors as
//     X_k = h_k sum_j (x_j h_j) g_{k-j},  h_m = exp(dir pi i m^2 / n),  g = conj(h),
// a linear convolution of a_j = x_j h_j (j < n) with g over -(n-1)..(n-1).
// It is computed as a cyclic convolution of length M = the smallest power
// of two >= 2n - 1: the chirp is stored wrapped (g_m at m and at M - m),
// its transform G = FFT_M(g) / M is a per-(n, dir) table, and each batch is
//     a = x h (zero-padded to M)  ->  A = FFT_M(a)  ->  A G  ->  c = IFFT_M(A G)
//     ->  X_k = h_k c_k, k < n.
// The phase m^2 / n is reduced modulo 2 in exact integer arithmetic
// (m^2 mod 2n) before the float64 sine and cosine, so the chirp keeps its
// accuracy for large m.  G is computed once on the host in float64 (an
// iterative radix-2 FFT) and rounded to float32, like the twiddle tables;
// the data never leaves the GPU.
//
// For 32 <= M <= 8192 (and no caller plan) the whole chain is one kernel,
// one signal per M/16 threads: the chirp product is formed as the signal is
// loaded, the forward M-point transform (the compile-time radix-16 stage
// schedule) writes its output times G into the shared-memory exchange
// buffer, the inverse transform reads it back and its last stage writes
// h_k c_k for k < n straight to global memory.  HBM then carries 16 bytes
// per element, as for a power-of-two length.  Otherwise (or with a plan for
// the M-point transforms) the chain runs as three elementwise kernels and
// two batched FFT launches through a scratch buffer.
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "fft_common.cuh"
#include "internal.h"

namespace bplg {

namespace {

constexpr int kFusedMinLog = 5, kFusedMaxLog = 13;  // at most 512 threads: 128 registers each

// The fused chain for M = 2^LOGM (radix 16, padded interleaved exchange).
template <int LOGM>
__global__ void __launch_bounds__(512)
    bluestein_fused_kernel(const float2 *__restrict__ x, float2 *__restrict__ X, const float2 *__restrict__ h,
                           const float2 *__restrict__ G, const float2 *__restrict__ tw, int64_t n, int spb,
                           int64_t batch) {
    using S = FftShape<16, LOGM>;
    constexpr int M = 1 << LOGM;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x;
    const int s = tid >> S::LOGT;
    const int j = tid & (S::T - 1);
    const int64_t sig = static_cast<int64_t>(blockIdx.x) * spb + s;
    const bool active = sig < batch;
    float2 *buf2 = reinterpret_cast<float2 *>(smem_raw) + s * sig_stride<0, 1>(M);
    float *buf1 = reinterpret_cast<float *>(buf2);
    const float2 *xs = x + sig * n;
    float2 v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const int e = j + m * S::T;
        v[m] = active && e < n ? cmul(__ldcs(xs + e), __ldg(h + e)) : make_float2(0.f, 0.f);
    }
    // forward transform; its output times G goes to the exchange buffer
    auto to_smem = [&](int pos, float2 val) { buf2[pad_g<16>(pos)] = cmul(val, __ldg(G + pos)); };
    fft_fixed_stages_st<16, LOGM, -1, 0, 0, true>(v, buf2, buf1, j, tw, to_smem);
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = buf2[pad_g<16>(j + m * S::T)];
    // inverse transform; X_k = h_k c_k for k < n
    float2 *Xs = X + sig * n;
    auto to_out = [&](int pos, float2 val) {
        if (active && pos < n) __stcs(Xs + pos, cmul(val, __ldg(h + pos)));
    };
    fft_fixed_stages_st<16, LOGM, 1, 0, 0, true>(v, buf2, buf1, j, tw, to_out);
}

const void *fused_func(int logm) {
    switch (logm) {
        case 5: return reinterpret_cast<const void *>(&bluestein_fused_kernel<5>);
        case 6: return reinterpret_cast<const void *>(&bluestein_fused_kernel<6>);
        case 7: return reinterpret_cast<const void *>(&bluestein_fused_kernel<7>);
        case 8: return reinterpret_cast<const void *>(&bluestein_fused_kernel<8>);
        case 9: return reinterpret_cast<const void *>(&bluestein_fused_kernel<9>);
        case 10: return reinterpret_cast<const void *>(&bluestein_fused_kernel<10>);
        case 11: return reinterpret_cast<const void *>(&bluestein_fused_kernel<11>);
        case 12: return reinterpret_cast<const void *>(&bluestein_fused_kernel<12>);
        case 13: return reinterpret_cast<const void *>(&bluestein_fused_kernel<13>);
        default: return nullptr;
    }
}

// a[s][j] = x[s][j] h_j for j < n, 0 for n <= j < M
__global__ void bluestein_pre(const float2 *__restrict__ x, float2 *__restrict__ a, const float2 *__restrict__ h,
                              int64_t n, int logm, int64_t total) {
    const int64_t m_mask = (int64_t(1) << logm) - 1;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t s = i >> logm, j = i & m_mask;
        a[i] = j < n ? cmul(__ldcs(x + s * n + j), h[j]) : make_float2(0.f, 0.f);
    }
}

// A[s][k] *= G[k]
__global__ void bluestein_mul(float2 *__restrict__ A, const float2 *__restrict__ G, int logm, int64_t total) {
    const int64_t m_mask = (int64_t(1) << logm) - 1;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        A[i] = cmul(A[i], G[i & m_mask]);
}

// X[s][k] = h_k c[s][k] for k < n
__global__ void bluestein_post(const float2 *__restrict__ c, float2 *__restrict__ X, const float2 *__restrict__ h,
                               int64_t n, int logm, int64_t total) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t s = i / n, k = i - s * n;
        __stcs(X + i, cmul(c[(s << logm) + k], h[k]));
    }
}

// in-place iterative radix-2 FFT in float64, exp(-2 pi i jk / M)
void host_fft(std::vector<double> &re, std::vector<double> &im) {
    const size_t M = re.size();
    for (size_t i = 1, j = 0; i < M; ++i) {  // bit reversal
        size_t bit = M >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            std::swap(re[i], re[j]);
            std::swap(im[i], im[j]);
        }
    }
    for (size_t len = 2; len <= M; len <<= 1) {
        const size_t half = len >> 1;
        std::vector<double> wr(half), wi(half);
        for (size_t k = 0; k < half; ++k) {
            const double ang = -2.0 * M_PI * static_cast<double>(k) / static_cast<double>(len);
            wr[k] = std::cos(ang);
            wi[k] = std::sin(ang);
        }
        for (size_t i = 0; i < M; i += len)
            for (size_t k = 0; k < half; ++k) {
                const double ur = re[i + k], ui = im[i + k];
                const double vr = re[i + k + half] * wr[k] - im[i + k + half] * wi[k];
                const double vi = re[i + k + half] * wi[k] + im[i + k + half] * wr[k];
                re[i + k] = ur + vr;
                im[i + k] = ui + vi;
                re[i + k + half] = ur - vr;
                im[i + k + half] = ui - vi;
            }
    }
}

struct Tables {
    float2 *h = nullptr;  // n entries
    float2 *G = nullptr;  // M entries
};

std::mutex g_mu;
std::map<std::tuple<int, int64_t, int>, Tables> g_tables;  // (device, n, dir)

int tables_for(int64_t n, int dir, int logm, Tables *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_tables.find(std::make_tuple(dev, n, dir));
    if (it != g_tables.end()) {
        *out = it->second;
        return BPLG_OK;
    }
    const int64_t M = int64_t(1) << logm;
    // chirp h_m = exp(dir pi i (m^2 mod 2n) / n) in float64
    std::vector<double> hr(n), hi(n);
    for (int64_t m = 0; m < n; ++m) {
        const int64_t q = (m * m) % (2 * n);  // m < 2^23: m^2 < 2^46
        const double ang = dir * M_PI * static_cast<double>(q) / static_cast<double>(n);
        hr[m] = std::cos(ang);
        hi[m] = std::sin(ang);
    }
    // g = conj(h) wrapped to length M, its transform / M
    std::vector<double> gr(M, 0.0), gi(M, 0.0);
    for (int64_t m = 0; m < n; ++m) {
        gr[m] = hr[m];
        gi[m] = -hi[m];
        if (m > 0) {
            gr[M - m] = hr[m];
            gi[M - m] = -hi[m];
        }
    }
    host_fft(gr, gi);
    std::vector<float2> h32(n), G32(M);
    for (int64_t m = 0; m < n; ++m) h32[m] = make_float2(static_cast<float>(hr[m]), static_cast<float>(hi[m]));
    const double inv = 1.0 / static_cast<double>(M);
    for (int64_t k = 0; k < M; ++k)
        G32[k] = make_float2(static_cast<float>(gr[k] * inv), static_cast<float>(gi[k] * inv));
    Tables t;
    if ((e = cudaMalloc(&t.h, n * sizeof(float2))) != cudaSuccess) return cuda_error(e, "Bluestein tables");
    if ((e = cudaMalloc(&t.G, M * sizeof(float2))) != cudaSuccess) {
        cudaFree(t.h);
        return cuda_error(e, "Bluestein tables");
    }
    if ((e = cudaMemcpy(t.h, h32.data(), n * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(t.G, G32.data(), M * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess) {
        cudaFree(t.h);
        cudaFree(t.G);
        return cuda_error(e, "Bluestein tables upload");
    }
    g_tables[std::make_tuple(dev, n, dir)] = t;
    *out = t;
    return BPLG_OK;
}

int elementwise_grid(int64_t total) {
    const int64_t blocks = (total + 255) / 256;
    return static_cast<int>(blocks < 152 * 16 ? blocks : 152 * 16);
}

}  // namespace

int fft_bluestein_launch(const bplg_plan *plan_m, const void *in, void *out, int64_t n, int64_t batch, int dir,
                         cudaStream_t s) {
    if (n < 2 || n > (int64_t(1) << kBluesteinMaxLog))
        return set_error(BPLG_ERR_UNSUPPORTED_SIZE, "fft: n must be in [2, 2^23] when it is not a power of two");
    const int64_t M = next_pow2(2 * n - 1);
    const int logm = ilog2(M);
    Tables t;
    int rc = tables_for(n, dir, logm, &t);
    if (rc != BPLG_OK) return rc;
    if (!plan_m && logm >= kFusedMinLog && logm <= kFusedMaxLog) {
        const void *tw = nullptr;
        rc = twiddles_for_current_device(&tw);
        if (rc != BPLG_OK) return rc;
        const void *f = fused_func(logm);
        const int T = static_cast<int>(M / 16);
        int spb = T >= 256 ? 1 : 256 / T;  // 256 or 512 threads per block
        const int smem = spb * sig_stride<0, 1>(static_cast<int>(M)) * static_cast<int>(sizeof(float2));
        rc = ensure_smem_attr(f, smem);
        if (rc != BPLG_OK) return rc;
        const int64_t blocks = (batch + spb - 1) / spb;
        rc = check_grid(blocks, "fft (Bluestein)");
        if (rc != BPLG_OK) return rc;
        const float2 *xi = static_cast<const float2 *>(in);
        float2 *xo = static_cast<float2 *>(out);
        void *args[] = {(void *)&xi, (void *)&xo, (void *)&t.h, (void *)&t.G, (void *)&tw, &n, &spb, &batch};
        cudaError_t e = cudaLaunchKernel(f, dim3(static_cast<unsigned>(blocks)), dim3(T * spb), args,
                                         static_cast<size_t>(smem), s);
        return e == cudaSuccess ? BPLG_OK : launch_error(e, "Bluestein fused launch", f, blocks, T * spb, smem);
    }
    // the inner transforms' plan: the caller's (made for M) or the default
    bplg_plan pm;
    if (plan_m) {
        if (plan_m->op != BPLG_OP_FFT || plan_m->n != M)
            return set_error(BPLG_ERR_INVALID_PLAN, "fft: a length that is not a power of two takes a plan for the "
                                                    "inner power-of-two length M = next_pow2(2n - 1), or NULL");
        pm = *plan_m;
        std::string why;
        rc = check_plan_on_device(pm, BPLG_F32, M, &why);
        if (rc == BPLG_ERR_INVALID_PLAN) return set_error(rc, "invalid plan: " + why);
        if (rc != BPLG_OK) return rc;
    } else {
        rc = bplg_query_plan(BPLG_OP_FFT, BPLG_F32, M, batch, &pm);
        if (rc != BPLG_OK) return rc;
    }
    void *scr = nullptr;
    rc = stream_scratch(kScratchBluestein, static_cast<size_t>(M) * static_cast<size_t>(batch) * sizeof(float2), s, &scr);
    if (rc != BPLG_OK) return rc;
    float2 *a = static_cast<float2 *>(scr);
    const int64_t total_m = M * batch, total_n = n * batch;
    bluestein_pre<<<elementwise_grid(total_m), 256, 0, s>>>(static_cast<const float2 *>(in), a, t.h, n, logm, total_m);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "Bluestein pre-multiply");
    rc = fft_launch(pm, a, a, M, batch, -1, s);
    if (rc != BPLG_OK) return rc;
    bluestein_mul<<<elementwise_grid(total_m), 256, 0, s>>>(a, t.G, logm, total_m);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "Bluestein product");
    rc = fft_launch(pm, a, a, M, batch, +1, s);
    if (rc != BPLG_OK) return rc;
    bluestein_post<<<elementwise_grid(total_n), 256, 0, s>>>(a, static_cast<float2 *>(out), t.h, n, logm, total_n);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "Bluestein post-multiply");
    return BPLG_OK;
}

}  // namespace bplg
