// Size-specialised batched Stockham FFT kernel (same plan, same arithmetic,
// same shared-memory layout as fft_kernel) for padded, directly loaded
// transforms of radix 8 or 16; its compile-time stage schedule
// (fft_fixed_stages) is described in fft_common.cuh.  Instantiated per
// direction in fft_fixed_fwd.cu and fft_fixed_inv.cu, which compile in
// parallel: radix 16 for n = 2^5 .. 2^14, radix 8 for n = 2^4 .. 2^9.
#pragma once

#include "device_util.cuh"
#include "fft_common.cuh"

namespace bplg {

template <int R, int LOGN, int DIR, int LAYOUT, int MAXT>
__global__ void __launch_bounds__(MAXT)
    fft_fixed_kernel(const float2 *in, float2 *out, const float2 *__restrict__ tw, int logn, int spb,
                     int64_t batch) {
    using S = FftShape<R, LOGN>;
    (void)logn;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x;
    const int s = tid >> S::LOGT;
    const int j = tid & (S::T - 1);
    const int64_t sig = static_cast<int64_t>(blockIdx.x) * spb + s;
    const bool active = sig < batch;
    const int sbase = s * sig_stride<LAYOUT, 1>(1 << LOGN);
    float2 *buf2 = reinterpret_cast<float2 *>(smem_raw) + sbase;
    float *buf1 = reinterpret_cast<float *>(smem_raw) + sbase;
    const float2 *g = in + sig * (int64_t(1) << LOGN) + j;
    float2 v[R];
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = active ? __ldcs(g + m * S::T) : make_float2(0.f, 0.f);
    fft_fixed_stages<R, LOGN, DIR, LAYOUT, 0>(v, buf2, buf1, j, tw, out + sig * (int64_t(1) << LOGN), active);
}

// Blocks of up to 512 threads get 128 registers per thread (the radix-16
// sizes from 2^10 on need about 60 and have both bounds); smaller sizes use
// the 1024-thread bound only.
template <int DIR>
const void *fft_fixed_lookup_dir(int radix, int layout, int threads, int logn) {
#define BPLG_FIXED(R, L, LAY, T) reinterpret_cast<const void *>(&fft_fixed_kernel<R, L, DIR, LAY, T>)
#define BPLG_FIXED_SIZES16(LAY, T)                                                                  \
    switch (logn) {                                                                                 \
        case 10: return BPLG_FIXED(16, 10, LAY, T);                                                 \
        case 11: return BPLG_FIXED(16, 11, LAY, T);                                                 \
        case 12: return BPLG_FIXED(16, 12, LAY, T);                                                 \
        case 13: return BPLG_FIXED(16, 13, LAY, T);                                                 \
        case 14: return BPLG_FIXED(16, 14, LAY, T);                                                 \
        default: break;                                                                             \
    }
    if (layout < 0 || layout > 1) return nullptr;
    if (radix == 16) {
        if (logn >= 10) {
            if (threads <= 512) {
                if (layout == 0) { BPLG_FIXED_SIZES16(0, 512) } else { BPLG_FIXED_SIZES16(1, 512) }
            } else {
                if (layout == 0) { BPLG_FIXED_SIZES16(0, 1024) } else { BPLG_FIXED_SIZES16(1, 1024) }
            }
            return nullptr;
        }
        switch (logn * 2 + layout) {
            case 10: return BPLG_FIXED(16, 5, 0, 1024);
            case 11: return BPLG_FIXED(16, 5, 1, 1024);
            case 12: return BPLG_FIXED(16, 6, 0, 1024);
            case 13: return BPLG_FIXED(16, 6, 1, 1024);
            case 14: return BPLG_FIXED(16, 7, 0, 1024);
            case 15: return BPLG_FIXED(16, 7, 1, 1024);
            case 16: return BPLG_FIXED(16, 8, 0, 1024);
            case 17: return BPLG_FIXED(16, 8, 1, 1024);
            case 18: return BPLG_FIXED(16, 9, 0, 1024);
            case 19: return BPLG_FIXED(16, 9, 1, 1024);
            default: return nullptr;
        }
    }
    if (radix == 8) {
        switch (logn * 2 + layout) {
            case 8: return BPLG_FIXED(8, 4, 0, 1024);
            case 9: return BPLG_FIXED(8, 4, 1, 1024);
            case 10: return BPLG_FIXED(8, 5, 0, 1024);
            case 11: return BPLG_FIXED(8, 5, 1, 1024);
            case 12: return BPLG_FIXED(8, 6, 0, 1024);
            case 13: return BPLG_FIXED(8, 6, 1, 1024);
            case 14: return BPLG_FIXED(8, 7, 0, 1024);
            case 15: return BPLG_FIXED(8, 7, 1, 1024);
            case 16: return BPLG_FIXED(8, 8, 0, 1024);
            case 17: return BPLG_FIXED(8, 8, 1, 1024);
            case 18: return BPLG_FIXED(8, 9, 0, 1024);
            case 19: return BPLG_FIXED(8, 9, 1, 1024);
            default: return nullptr;
        }
    }
    return nullptr;
#undef BPLG_FIXED_SIZES16
#undef BPLG_FIXED
}

}  // namespace bplg
