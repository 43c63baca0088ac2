// Mixed-radix FFT kernels, shard 0 of kMixedShards (lengths kLengths.v[0],
// kLengths.v[0 + kMixedShards], ...): see fft_mixed.cuh.
#include "fft_mixed.cuh"

namespace bplg {
bool mixed_shard_0(int n, int dir, MixedLaunch *o) { return mixed_shard<0>(n, dir, o); }
}  // namespace bplg
