// Size-specialised batched FFT kernels, forward direction (see fft_fixed.cuh).
#include "fft_fixed.cuh"

namespace bplg {

const void *fft_fixed_lookup_fwd(int radix, int layout, int threads, int logn) {
    return fft_fixed_lookup_dir<-1>(radix, layout, threads, logn);
}

}  // namespace bplg
