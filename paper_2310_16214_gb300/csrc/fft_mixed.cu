// Host side of the mixed-radix FFT: the twiddle table of each length and the
// launch of its compile-time kernel (fft_mixed.cuh; the kernels are spread
// over the translation units fft_mixed_s0.cu .. fft_mixed_s7.cu).
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fft_mixed.cuh"
#include "internal.h"

namespace bplg {

static_assert(kMixedMaxN == kMixedMaxLen, "one limit for the mixed-radix lengths");

namespace {

std::mutex g_mu;
std::map<std::pair<int, int64_t>, float2 *> g_tables;  // (device, n) -> exp(-2 pi i e / n), e < n

int table_for(int64_t n, const float2 **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_tables.find(std::make_pair(dev, n));
    if (it != g_tables.end()) {
        *out = it->second;
        return BPLG_OK;
    }
    std::vector<float2> h(static_cast<size_t>(n));
    for (int64_t k = 0; k < n; ++k) {
        const double ang = -2.0 * M_PI * static_cast<double>(k) / static_cast<double>(n);
        h[static_cast<size_t>(k)] = make_float2(static_cast<float>(std::cos(ang)), static_cast<float>(std::sin(ang)));
    }
    float2 *d = nullptr;
    if ((e = cudaMalloc(&d, static_cast<size_t>(n) * sizeof(float2))) != cudaSuccess)
        return cuda_error(e, "mixed-radix twiddles");
    if ((e = cudaMemcpy(d, h.data(), static_cast<size_t>(n) * sizeof(float2), cudaMemcpyHostToDevice)) !=
        cudaSuccess) {
        cudaFree(d);
        return cuda_error(e, "mixed-radix twiddles upload");
    }
    g_tables[std::make_pair(dev, n)] = d;
    *out = d;
    return BPLG_OK;
}

bool (*const kShards[kMixedShards])(int, int, MixedLaunch *) = {
    mixed_shard_0, mixed_shard_1, mixed_shard_2, mixed_shard_3,
    mixed_shard_4, mixed_shard_5, mixed_shard_6, mixed_shard_7};

bool lookup(int64_t n, int dir, MixedLaunch *o) {
    if (!mixed_detail::has_kernel(static_cast<int>(n))) return false;
    for (auto f : kShards)
        if (f(static_cast<int>(n), dir, o)) return true;
    return false;
}

}  // namespace

bool fft_mixed_supported(int64_t n) { return n > 2 && n <= kMixedMaxN && mixed_detail::has_kernel(static_cast<int>(n)); }

int fft_mixed_launch(const void *in, void *out, int64_t n, int64_t batch, int dir, cudaStream_t s) {
    MixedLaunch ml{};
    if (!fft_mixed_supported(n) || !lookup(n, dir, &ml))
        return set_error(BPLG_ERR_UNSUPPORTED_SIZE, "fft (mixed radix): n must be 2^a 3^b 5^c, not a power of two, "
                                                    "at most " + std::to_string(kMixedMaxN));
    const float2 *tw = nullptr;
    int rc = table_for(n, &tw);
    if (rc != BPLG_OK) return rc;
    rc = ensure_smem_attr(ml.fn, ml.smem);
    if (rc != BPLG_OK) return rc;
    const int64_t blocks = (batch + ml.spb - 1) / ml.spb;
    rc = check_grid(blocks, "fft (mixed radix)");
    if (rc != BPLG_OK) return rc;
    const float2 *xi = static_cast<const float2 *>(in);
    float2 *xo = static_cast<float2 *>(out);
    void *args[] = {(void *)&xi, (void *)&xo, (void *)&tw, &batch};
    cudaError_t e = cudaLaunchKernel(ml.fn, dim3(static_cast<unsigned>(blocks)), dim3(ml.threads), args,
                                     static_cast<size_t>(ml.smem), s);
    return e == cudaSuccess ? BPLG_OK : launch_error(e, "fft (mixed radix) launch", ml.fn, blocks, ml.threads, ml.smem);
}

}  // namespace bplg
