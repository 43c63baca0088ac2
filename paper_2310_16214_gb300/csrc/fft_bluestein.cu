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
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.h"

namespace bplg {

namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
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
