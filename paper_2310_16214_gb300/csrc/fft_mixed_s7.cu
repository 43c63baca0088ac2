// Mixed-radix FFT kernels, shard 7 of kMixedShards (lengths kLengths.v[7],
// kLengths.v[7 + kMixedShards], ...): see fft_mixed.cuh.
#include "fft_mixed.cuh"

namespace bplg {
bool mixed_shard_7(int n, int dir, MixedLaunch *o) { return mixed_shard<7>(n, dir, o); }
}  // namespace bplg
