// Mixed-radix FFT kernels, shard 4 of kMixedShards (lengths kLengths.v[4],
// kLengths.v[4 + kMixedShards], ...): see fft_mixed.cuh.
#include "fft_mixed.cuh"

namespace bplg {
bool mixed_shard_4(int n, int dir, MixedLaunch *o) { return mixed_shard<4>(n, dir, o); }
}  // namespace bplg
