// Mixed-radix FFT kernels, shard 1 of kMixedShards (lengths kLengths.v[1],
// kLengths.v[1 + kMixedShards], ...): see fft_mixed.cuh.
#include "fft_mixed.cuh"

namespace bplg {
bool mixed_shard_1(int n, int dir, MixedLaunch *o) { return mixed_shard<1>(n, dir, o); }
}  // namespace bplg
