// Mixed-radix FFT kernels, shard 2 of kMixedShards (lengths kLengths.v[2],
// kLengths.v[2 + kMixedShards], ...): see fft_mixed.cuh.
#include "fft_mixed.cuh"

namespace bplg {
bool mixed_shard_2(int n, int dir, MixedLaunch *o) { return mixed_shard<2>(n, dir, o); }
}  // namespace bplg
