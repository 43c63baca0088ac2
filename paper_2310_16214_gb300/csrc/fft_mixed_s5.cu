// Mixed-radix FFT kernels, shard 5 of kMixedShards (lengths kLengths.v[5],
// kLengths.v[5 + kMixedShards], ...): see fft_mixed.cuh.
#include "fft_mixed.cuh"

namespace bplg {
bool mixed_shard_5(int n, int dir, MixedLaunch *o) { return mixed_shard<5>(n, dir, o); }
}  // namespace bplg
