// Mixed-radix FFT kernels, shard 6 of kMixedShards (lengths kLengths.v[6],
// kLengths.v[6 + kMixedShards], ...): see fft_mixed.cuh.
#include "fft_mixed.cuh"

namespace bplg {
bool mixed_shard_6(int n, int dir, MixedLaunch *o) { return mixed_shard<6>(n, dir, o); }
}  // namespace bplg
