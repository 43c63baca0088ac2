// Mixed-radix FFT kernels, shard 3 of kMixedShards (lengths kLengths.v[3],
// kLengths.v[3 + kMixedShards], ...): see fft_mixed.cuh.
#include "fft_mixed.cuh"

namespace bplg {
bool mixed_shard_3(int n, int dir, MixedLaunch *o) { return mixed_shard<3>(n, dir, o); }
}  // namespace bplg
