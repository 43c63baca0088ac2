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

}  // extern "C"
