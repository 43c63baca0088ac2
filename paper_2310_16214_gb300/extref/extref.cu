// External references for the benchmark: the vendor libraries' versions of
// the three batched operations, timed beside this library on the same GPU.
// Measurement only; nothing in libbplg calls them, and they are built into a
// separate library (libbplg_extref.so).
//
//   extref_scan_bykey   CUB DeviceScan::InclusiveSumByKey over the whole batch,
//                       the key of element i being its signal i / n
//   extref_scan_each    CUB DeviceScan::InclusiveSum called once per signal
//                       (how a batch of independent scans is usually run
//                       with a library that has no batched scan)
//   extref_fft_c2c      cuFFT cufftPlanMany C2C, unnormalised, plan cached
//   extref_gtsv2        cuSPARSE gtsv2StridedBatch (x holds d on entry)
//   extref_fp64_fma     the FP64 pipe's measured throughput: independent
//                       chains of double-precision fused multiply-adds on
//                       every SM, timed with CUDA events (the denominator of
//                       the refined solve's roofline)
//
// Every function returns 0 on success, else a negative code: -1 bad argument,
// -2 CUDA error, -3 cuFFT error, -4 cuSPARSE error.  The scans take a caller
// workspace: called with temp == NULL they store the bytes needed in
// *temp_bytes and return 0.
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>

#include <cub/device/device_scan.cuh>
#include <cufft.h>
#include <cusparse.h>
#include <thrust/iterator/counting_iterator.h>
#include <thrust/iterator/transform_iterator.h>

namespace {

struct SignalOf {
    int64_t n;
    __host__ __device__ int64_t operator()(int64_t i) const { return i / n; }
};

template <typename T>
int scan_bykey(const T *in, T *out, int64_t n, int64_t batch, void *temp, size_t *temp_bytes, cudaStream_t s) {
    auto keys = thrust::make_transform_iterator(thrust::counting_iterator<int64_t>(0), SignalOf{n});
    const int64_t total = n * batch;
    cudaError_t e = cub::DeviceScan::InclusiveSumByKey(temp, *temp_bytes, keys, in, out, total,
                                                       ::cuda::std::equal_to<>(), s);
    return e == cudaSuccess ? 0 : -2;
}

template <typename T>
int scan_each(const T *in, T *out, int64_t n, int64_t batch, void *temp, size_t *temp_bytes, cudaStream_t s) {
    if (!temp) {
        cudaError_t e = cub::DeviceScan::InclusiveSum(nullptr, *temp_bytes, in, out, n, s);
        return e == cudaSuccess ? 0 : -2;
    }
    for (int64_t b = 0; b < batch; ++b) {
        size_t bytes = *temp_bytes;
        cudaError_t e = cub::DeviceScan::InclusiveSum(temp, bytes, in + b * n, out + b * n, n, s);
        if (e != cudaSuccess) return -2;
    }
    return 0;
}

// Eight independent chains of x = x * a + b per thread, `iters` times each:
// 16 flop per thread per iteration, nothing else on the FP64 pipe.  The
// chains converge to b / (1 - a), so the values stay finite; the sum is
// stored so that nothing is removed as dead code.
__global__ void __launch_bounds__(256) fp64_fma_kernel(double *out, int64_t iters, double a, double b) {
    const double s = 1e-3 * static_cast<double>(threadIdx.x);
    double x0 = s, x1 = s + 1.0, x2 = s + 2.0, x3 = s + 3.0, x4 = s + 4.0, x5 = s + 5.0, x6 = s + 6.0,
           x7 = s + 7.0;
#pragma unroll 4
    for (int64_t i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b);
        x1 = fma(x1, a, b);
        x2 = fma(x2, a, b);
        x3 = fma(x3, a, b);
        x4 = fma(x4, a, b);
        x5 = fma(x5, a, b);
        x6 = fma(x6, a, b);
        x7 = fma(x7, a, b);
    }
    out[static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x] = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
}

std::mutex g_mu;
std::map<std::tuple<int, int64_t, int64_t>, cufftHandle> g_plans;  // (device, n, batch)
std::map<int, cusparseHandle_t> g_sparse;                           // device

}  // namespace

extern "C" {

int extref_scan_bykey(int dtype, const void *in, void *out, int64_t n, int64_t batch, void *temp,
                      size_t *temp_bytes, void *stream) {
    if (!temp_bytes || n < 1 || batch < 1) return -1;
    auto s = static_cast<cudaStream_t>(stream);
    if (dtype == 0)
        return scan_bykey(static_cast<const int32_t *>(in), static_cast<int32_t *>(out), n, batch, temp, temp_bytes, s);
    return scan_bykey(static_cast<const float *>(in), static_cast<float *>(out), n, batch, temp, temp_bytes, s);
}

int extref_scan_each(int dtype, const void *in, void *out, int64_t n, int64_t batch, void *temp,
                     size_t *temp_bytes, void *stream) {
    if (!temp_bytes || n < 1 || batch < 1) return -1;
    auto s = static_cast<cudaStream_t>(stream);
    if (dtype == 0)
        return scan_each(static_cast<const int32_t *>(in), static_cast<int32_t *>(out), n, batch, temp, temp_bytes, s);
    return scan_each(static_cast<const float *>(in), static_cast<float *>(out), n, batch, temp, temp_bytes, s);
}

int extref_fft_c2c(const void *in, void *out, int64_t n, int64_t batch, int dir, void *stream) {
    if (n < 1 || batch < 1 || n > (int64_t(1) << 30) || batch > (int64_t(1) << 30) || (dir != -1 && dir != 1))
        return -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -2;
    cufftHandle plan;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto key = std::make_tuple(dev, n, batch);
        auto it = g_plans.find(key);
        if (it == g_plans.end()) {
            int nn = static_cast<int>(n);
            if (cufftPlanMany(&plan, 1, &nn, nullptr, 1, nn, nullptr, 1, nn, CUFFT_C2C, static_cast<int>(batch)) !=
                CUFFT_SUCCESS)
                return -3;
            g_plans[key] = plan;
        } else {
            plan = it->second;
        }
    }
    if (cufftSetStream(plan, static_cast<cudaStream_t>(stream)) != CUFFT_SUCCESS) return -3;
    auto *i = const_cast<cufftComplex *>(static_cast<const cufftComplex *>(in));
    auto *o = static_cast<cufftComplex *>(out);
    return cufftExecC2C(plan, i, o, dir < 0 ? CUFFT_FORWARD : CUFFT_INVERSE) == CUFFT_SUCCESS ? 0 : -3;
}

int extref_gtsv2(const float *dl, const float *d, const float *du, float *x, int64_t n, int64_t batch, void *buffer,
                 size_t *bytes, void *stream) {
    if (!bytes || n < 3 || batch < 1 || n > (int64_t(1) << 30) || batch > (int64_t(1) << 30)) return -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -2;
    cusparseHandle_t h;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_sparse.find(dev);
        if (it == g_sparse.end()) {
            if (cusparseCreate(&h) != CUSPARSE_STATUS_SUCCESS) return -4;
            g_sparse[dev] = h;
        } else {
            h = it->second;
        }
    }
    if (cusparseSetStream(h, static_cast<cudaStream_t>(stream)) != CUSPARSE_STATUS_SUCCESS) return -4;
    const int m = static_cast<int>(n), bc = static_cast<int>(batch);
    if (!buffer) {
        return cusparseSgtsv2StridedBatch_bufferSizeExt(h, m, dl, d, du, x, bc, m, bytes) == CUSPARSE_STATUS_SUCCESS
                   ? 0
                   : -4;
    }
    return cusparseSgtsv2StridedBatch(h, m, dl, d, du, x, bc, m, buffer) == CUSPARSE_STATUS_SUCCESS ? 0 : -4;
}

// Throughput of the FP64 pipe: one launch of SMs x 8 blocks of 256 threads
// (full residency), each thread running eight chains of `iters` fused
// multiply-adds; the best of `reps` event-timed launches after one warm-up.
// *tflops = 16 * threads * iters / time.
int extref_fp64_fma(int64_t iters, int reps, double *tflops, double *best_ms, void *stream) {
    if (!tflops || !best_ms || iters < 1 || reps < 1) return -1;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -2;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -2;
    const int threads = 256, blocks = sms * 8;
    auto s = static_cast<cudaStream_t>(stream);
    double *out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) return -2;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int rc = 0;
    for (int r = 0; r <= reps && rc == 0; ++r) {
        cudaEventRecord(e0, s);
        fp64_fma_kernel<<<blocks, threads, 0, s>>>(out, iters, 0.999999, 1e-6);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = -2;
        float ms = 0.f;
        if (rc == 0 && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = -2;
        if (rc == 0 && r > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (rc != 0) return rc;
    *best_ms = best;
    *tflops = 16.0 * double(blocks) * threads * double(iters) / (best * 1e-3) / 1e12;
    return 0;
}

}  // extern "C"
