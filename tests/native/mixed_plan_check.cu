// Host-side check of the mixed-radix FFT planner (fft_mixed.cuh), built with
// nvcc and run without a GPU.  For every length with a kernel: the radices
// come from the allowed set in non-increasing order and multiply to n; the
// stage count is the least possible (a dynamic program over the divisors of
// n, independent of the planner's search); every stage's butterflies fit
// the threads (at most b a thread); the block fits the hardware limits
// (1024 threads, the opt-in shared memory, 2048 threads an SM); and the
// list of lengths is exactly the 2^a 3^b 5^c in [3, 12288] that are not
// powers of two.  Prints "OK <count>" or the first failure.
#include <cstdio>
#include <vector>

#include "fft_mixed.cuh"

using namespace bplg;
using namespace bplg::mixed_detail;

static const int kAllowed[] = {16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};

// least number of allowed radices whose product is n (0 for n = 1)
static int least_stages(int n, std::vector<int> &memo) {
    if (n == 1) return 0;
    if (memo[n] >= 0) return memo[n];
    int best = 1 << 20;
    for (int r : kAllowed)
        if (n % r == 0) {
            const int k = 1 + least_stages(n / r, memo);
            if (k < best) best = k;
        }
    memo[n] = best;
    return best;
}

static bool expected_length(int n) {
    if (n < 3 || (n & (n - 1)) == 0) return false;
    int v = n;
    for (int p : {2, 3, 5})
        while (v % p == 0) v /= p;
    return v == 1;
}

int main() {
    std::vector<int> memo(kMixedMaxLen + 1, -1);
    int count = 0, li = 0;
    for (int n = 1; n <= kMixedMaxLen; ++n) {
        if (expected_length(n) != has_kernel(n)) {
            printf("FAIL has_kernel(%d)\n", n);
            return 1;
        }
        if (!expected_length(n)) continue;
        ++count;
        if (li >= kNumLengths || kLengths.v[li++] != n) {
            printf("FAIL length list at %d\n", n);
            return 1;
        }
        const Plan p = mixed_plan(n);
        long prod = 1;
        int prev = 1 << 20;
        for (int s = 0; s < p.k; ++s) {
            bool ok = false;
            for (int r : kAllowed) ok = ok || r == p.r[s];
            if (!ok || p.r[s] > prev) {
                printf("FAIL n=%d radix %d at stage %d\n", n, p.r[s], s);
                return 1;
            }
            prev = p.r[s];
            prod *= p.r[s];
        }
        if (prod != n) {
            printf("FAIL n=%d radices multiply to %ld\n", n, prod);
            return 1;
        }
        if (p.k != least_stages(n, memo)) {
            printf("FAIL n=%d %d stages, %d possible\n", n, p.k, least_stages(n, memo));
            return 1;
        }
        int vmax = 0;
        for (int s = 0; s < p.k; ++s) {
            const int nb = n / p.r[s];
            const int bs = (nb + p.t - 1) / p.t;
            if (bs > p.b) {
                printf("FAIL n=%d stage %d needs %d butterflies a thread, plan says %d\n", n, s, bs, p.b);
                return 1;
            }
            vmax = bs * p.r[s] > vmax ? bs * p.r[s] : vmax;
        }
        const int smem = p.k > 1 ? (p.dbl ? 2 : 1) * p.spb * n * 8 : 0;
        if (vmax != p.vmax || p.t < 1 || p.t > 1024 || p.spb < 1 || p.threads < p.spb * p.t ||
            p.threads % 32 != 0 || p.threads > 1024 || smem > 232448 || p.minb < 1 ||
            p.minb * p.threads > 2048) {
            printf("FAIL n=%d shape t=%d spb=%d threads=%d minb=%d vmax=%d/%d smem=%d\n", n, p.t, p.spb, p.threads,
                   p.minb, p.vmax, vmax, smem);
            return 1;
        }
    }
    if (count != kNumLengths) {
        printf("FAIL %d lengths, table holds %d\n", count, kNumLengths);
        return 1;
    }
    printf("OK %d\n", count);
    return 0;
}
