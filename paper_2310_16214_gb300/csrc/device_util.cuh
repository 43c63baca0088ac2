// Device helpers shared by the library's kernels: streaming vector loads and
// stores, and the warp-shuffle prefix circuits of Fig. 1(d)/(f).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bplg {

constexpr unsigned kFullMask = 0xffffffffu;

// ---- streaming 16-byte accesses (data is touched once: evict-first)
__device__ __forceinline__ int4 ld_stream(const int4 *p) { return __ldcs(p); }
__device__ __forceinline__ float4 ld_stream(const float4 *p) { return __ldcs(p); }
__device__ __forceinline__ void st_stream(int4 *p, int4 v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(float4 *p, float4 v) { __stcs(p, v); }

template <typename T>
struct Vec4Of;
template <>
struct Vec4Of<int32_t> {
    using type = int4;
};
template <>
struct Vec4Of<float> {
    using type = float4;
};

template <typename T>
__device__ __forceinline__ T from_bits(uint32_t u);
template <>
__device__ __forceinline__ int32_t from_bits<int32_t>(uint32_t u) { return static_cast<int32_t>(u); }
template <>
__device__ __forceinline__ float from_bits<float>(uint32_t u) { return __uint_as_float(u); }
__device__ __forceinline__ uint32_t to_bits(int32_t v) { return static_cast<uint32_t>(v); }
__device__ __forceinline__ uint32_t to_bits(float v) { return __float_as_uint(v); }

// Load P consecutive elements (P a power of two, p aligned to min(16, 4P) bytes).
template <typename T, int P>
__device__ __forceinline__ void load_run(const T *p, T (&v)[P]) {
    using V4 = typename Vec4Of<T>::type;
    if constexpr (P >= 4) {
#pragma unroll
        for (int q = 0; q < P / 4; ++q) {
            V4 w = ld_stream(reinterpret_cast<const V4 *>(p) + q);
            v[4 * q + 0] = w.x;
            v[4 * q + 1] = w.y;
            v[4 * q + 2] = w.z;
            v[4 * q + 3] = w.w;
        }
    } else if constexpr (P == 2) {
        uint2 w = __ldcs(reinterpret_cast<const uint2 *>(p));
        v[0] = from_bits<T>(w.x);
        v[1] = from_bits<T>(w.y);
    } else {
        v[0] = __ldcs(p);
    }
}

template <typename T, int P>
__device__ __forceinline__ void store_run(T *p, const T (&v)[P]) {
    using V4 = typename Vec4Of<T>::type;
    if constexpr (P >= 4) {
#pragma unroll
        for (int q = 0; q < P / 4; ++q) {
            V4 w;
            w.x = v[4 * q + 0];
            w.y = v[4 * q + 1];
            w.z = v[4 * q + 2];
            w.w = v[4 * q + 3];
            st_stream(reinterpret_cast<V4 *>(p) + q, w);
        }
    } else if constexpr (P == 2) {
        uint2 w;
        w.x = to_bits(v[0]);
        w.y = to_bits(v[1]);
        __stcs(reinterpret_cast<uint2 *>(p), w);
    } else {
        __stcs(p, v[0]);
    }
}

// ---- warp-level inclusive prefix sums over aligned segments of `width`
// lanes (width a power of two <= 32); every lane of the warp must call.
//
// Kogge-Stone (Fig. 1(f)): log2(width) steps, step d adds the value d lanes
// below.
template <typename T>
__device__ __forceinline__ T seg_scan_ks(T x, int lane_in_seg, int width) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        if (d >= width) break;
        T y = __shfl_up_sync(kFullMask, x, d, width);
        if (lane_in_seg >= d) x += y;
    }
    return x;
}

// Ladner-Fischer, depth-minimal member (Fig. 1(d)): at step k every lane in
// the upper half of each 2^(k+1)-lane group adds the last value of the lower
// half.
template <typename T>
__device__ __forceinline__ T seg_scan_lf(T x, int lane_in_seg, int width) {
#pragma unroll
    for (int k = 1; k < 32; k <<= 1) {
        if (k >= width) break;
        int src = (lane_in_seg & ~(2 * k - 1)) + k - 1;
        T y = __shfl_sync(kFullMask, x, src, width);
        if (lane_in_seg & k) x += y;
    }
    return x;
}

template <int PATTERN, typename T>
__device__ __forceinline__ T seg_scan(T x, int lane_in_seg, int width) {
    if constexpr (PATTERN == 0)
        return seg_scan_ks(x, lane_in_seg, width);
    else
        return seg_scan_lf(x, lane_in_seg, width);
}

}  // namespace bplg
