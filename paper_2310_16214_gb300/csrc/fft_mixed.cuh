// Mixed-radix Stockham FFT for lengths n = 2^a 3^b 5^c that are not powers
// of two (at most 12288), one kernel per length with its whole stage
// schedule fixed at compile time.  (The paper keeps to N = r^n; this extends
// the radix-r Stockham formulation of Section III to products of small
// radices, so such lengths need not go through Bluestein's identity.)
//
// Stockham autosort, decimation in time.  With n = r_1 r_2 ... r_K, after
// the stages r_1 .. r_{s-1} the array holds, for L = r_1 ... r_{s-1} and
// m = n / L, the L-point DFTs of the m decimated subsequences x[k + m t]
// (t < L): entry j of subsequence k at index j m + k.  Stage s (radix r,
// m' = m / r) joins subsequences k' + m' p (p < r) into the (L r)-point DFT
// of subsequence k': with j'' = j + L q,
//     A'[j + L q][k'] = sum_p W_r^(p q) (W_{L r}^(p j) A[j][k' + m' p]),
// read at j r m' + p m' + k' and written at (j + L q) m' + k'.  After the
// last stage L = n, m = 1 and the array is X in natural order.  W_m =
// exp(dir 2 pi i / m); every stage twiddle W_{L r}^(p j) = W_n^(p j m') is
// an entry of one n-point table, computed on the host in float64 and
// rounded to float32, like the power-of-two tables.
//
// Radices 16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2: the 3- and 5-point DFTs
// written out, the composite ones as two factors with their inner twiddles
// computed at compile time (float64 series, rounded once).  Because n, the
// radices and every stage's m' are compile-time constants, the index
// arithmetic folds into constants and immediates, and each kernel holds the
// code of its own radices only (so its registers are those of its largest
// codelet).  The plan (mixed_plan below): the fewest stages, radices in
// non-increasing order; T threads per signal, each doing at most B
// butterflies a stage (one in the smallest-radix stage unless n / r_min
// exceeds 1024 threads, or one in the largest-radix stage when the radices
// are at least a factor two apart); S
// signals a block and a register budget, chosen for small blocks and
// enough busy threads per SM.  The signals sit in one shared-memory buffer
// (n complex values each) -- a stage reads its inputs into registers, the
// block waits, and writes its outputs in place -- or in two that the stages
// alternate between, where that costs no block per SM; the first stage
// reads global memory and the last writes it.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <utility>

#include "fft_common.cuh"

namespace bplg {

constexpr int kMixedMaxLen = 12288;  // the largest length with a kernel
constexpr int kMixedShards = 8;      // translation units the kernels are spread over

namespace mixed_detail {

// cos and sin of 2 pi k / m at compile time, in double: the angle is
// reduced exactly (by the quadrant of 4k / m) to [0, pi / 2) and the
// Taylor series of sine and cosine summed there (24 terms: the remainder is
// below 1e-40 for arguments up to pi / 2)
constexpr double kPiD = 3.14159265358979323846264338327950288;
constexpr double taylor_sin(double x) {
    double t = x, sum = x;
    for (int i = 1; i < 24; ++i) {
        t *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
        sum += t;
    }
    return sum;
}
constexpr double taylor_cos(double x) {
    double t = 1.0, sum = 1.0;
    for (int i = 1; i < 24; ++i) {
        t *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
        sum += t;
    }
    return sum;
}
constexpr double cos_2pi(int k, int m) {
    const int kk = ((k % m) + m) % m;
    const int q = (4 * kk) / m, r = 4 * kk - q * m;  // angle = (q + r / m) pi / 2
    const double x = 0.5 * kPiD * r / m;
    return q == 0 ? taylor_cos(x) : q == 1 ? -taylor_sin(x) : q == 2 ? -taylor_cos(x) : taylor_sin(x);
}
constexpr double sin_2pi(int k, int m) {
    const int kk = ((k % m) + m) % m;
    const int q = (4 * kk) / m, r = 4 * kk - q * m;
    const double x = 0.5 * kPiD * r / m;
    return q == 0 ? taylor_sin(x) : q == 1 ? taylor_cos(x) : q == 2 ? -taylor_sin(x) : -taylor_cos(x);
}

// In-register 3- and 5-point DFTs, y_q = sum_p v_p exp(DIR 2 pi i p q / R).
// c_k = cos(2 pi k / R), s_k = sin(2 pi k / R).
template <int DIR>
__device__ __forceinline__ void dft3(float2 (&v)[3]) {
    constexpr float c1 = -0.5f, s1 = DIR * 0.86602540378443864676f;
    const float2 t = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    const float2 b = make_float2(fmaf(c1, t.x, v[0].x), fmaf(c1, t.y, v[0].y));
    const float2 e = make_float2(-s1 * d.y, s1 * d.x);  // i s1 d
    v[0] = cadd(v[0], t);
    v[1] = cadd(b, e);
    v[2] = csub(b, e);
}

template <int DIR>
__device__ __forceinline__ void dft5(float2 (&v)[5]) {
    constexpr float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;
    constexpr float s1 = DIR * 0.95105651629515357212f, s2 = DIR * 0.58778525229247312917f;
    const float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    const float2 d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
    const float2 b1 = make_float2(fmaf(c2, t2.x, fmaf(c1, t1.x, v[0].x)), fmaf(c2, t2.y, fmaf(c1, t1.y, v[0].y)));
    const float2 b2 = make_float2(fmaf(c1, t2.x, fmaf(c2, t1.x, v[0].x)), fmaf(c1, t2.y, fmaf(c2, t1.y, v[0].y)));
    // e1 = i (s1 d1 + s2 d2), e2 = i (s2 d1 - s1 d2)
    const float2 u1 = make_float2(fmaf(s2, d2.x, s1 * d1.x), fmaf(s2, d2.y, s1 * d1.y));
    const float2 u2 = make_float2(fmaf(-s1, d2.x, s2 * d1.x), fmaf(-s1, d2.y, s2 * d1.y));
    const float2 e1 = make_float2(-u1.y, u1.x), e2 = make_float2(-u2.y, u2.x);
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = cadd(b1, e1);
    v[4] = csub(b1, e1);
    v[2] = cadd(b2, e2);
    v[3] = csub(b2, e2);
}

template <int R, int DIR>
__device__ __forceinline__ void dft_any(float2 (&v)[R]);

// R = A B points as A B-point DFTs, twiddles W_R^(n1 k2), then B A-point
// DFTs (the two-factor Cooley-Tukey step): with n = n1 + A n2 and
// k = k2 + B k1, X[k] = sum_n1 W_A^(n1 k1) [W_R^(n1 k2) sum_n2 x[n] W_B^(n2 k2)]
template <int A, int B, int DIR>
__device__ __forceinline__ void dft_two_factor(float2 (&v)[A * B]) {
    float2 y[A][B];
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) {
        float2 u[B];
#pragma unroll
        for (int n2 = 0; n2 < B; ++n2) u[n2] = v[n1 + A * n2];
        dft_any<B, DIR>(u);
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) {
            if (n1 == 0 || k2 == 0) {
                y[n1][k2] = u[k2];
            } else {
                const float c = static_cast<float>(cos_2pi(n1 * k2, A * B));
                const float sn = static_cast<float>(DIR * sin_2pi(n1 * k2, A * B));
                y[n1][k2] = make_float2(u[k2].x * c - u[k2].y * sn, u[k2].x * sn + u[k2].y * c);
            }
        }
    }
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) {
        float2 w[A];
#pragma unroll
        for (int n1 = 0; n1 < A; ++n1) w[n1] = y[n1][k2];
        dft_any<A, DIR>(w);
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) v[k2 + B * k1] = w[k1];
    }
}

template <int R, int DIR>
__device__ __forceinline__ void dft_any(float2 (&v)[R]) {
    if constexpr (R == 3) {
        dft3<DIR>(v);
    } else if constexpr (R == 5) {
        dft5<DIR>(v);
    } else if constexpr (R == 6) {
        dft_two_factor<2, 3, DIR>(v);
    } else if constexpr (R == 9) {
        dft_two_factor<3, 3, DIR>(v);
    } else if constexpr (R == 10) {
        dft_two_factor<2, 5, DIR>(v);
    } else if constexpr (R == 12) {
        dft_two_factor<4, 3, DIR>(v);
    } else if constexpr (R == 15) {
        dft_two_factor<3, 5, DIR>(v);
    } else {
        dft_codelet<R, DIR>(v);
    }
}

// ---------------------------------------------------------------- plan

constexpr int kNumRadices = 11;
constexpr int kRadices[kNumRadices] = {16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};
constexpr int kMaxStages = 8;
constexpr int kMaxThreads = 1024;
constexpr int kSmemPerSm = 233472;    // shared memory of one SM available to blocks
constexpr int kSmemPerBlock = 232448; // the opt-in limit of one block

constexpr bool is_smooth(int n) {
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    while (n % 5 == 0) n /= 5;
    return n == 1;
}
constexpr bool has_kernel(int n) { return n >= 3 && n <= kMixedMaxLen && (n & (n - 1)) != 0 && is_smooth(n); }

struct Plan {
    int k = 0;                 // stages
    int r[kMaxStages] = {};    // radices, first stage first
    int b = 0;                 // most butterflies a thread does in one stage
    int t = 0;                 // threads per signal
    int spb = 0;               // signals per block
    int threads = 0;           // block size (spb t rounded up to whole warps)
    int minb = 0;              // blocks per SM the register budget is set for
    int vmax = 0;              // complex values a thread holds across a barrier
    bool dbl = false;          // two buffers a signal (one barrier a stage instead of two)
};

constexpr int rmin_of(const Plan &p) {
    int m = 1 << 30;
    for (int i = 0; i < p.k; ++i) m = p.r[i] < m ? p.r[i] : m;
    return m;
}
constexpr int rmax_of(const Plan &p) {
    int m = 0;
    for (int i = 0; i < p.k; ++i) m = p.r[i] > m ? p.r[i] : m;
    return m;
}
constexpr int bfly_per_thread(int n, int r_min) {
    const int most = n / r_min;  // butterflies of the smallest-radix stage
    return (most + kMaxThreads - 1) / kMaxThreads;
}
// a better than c: fewer stages, then fewer butterflies per thread, then a
// larger smallest radix (stages closer in size, fewer idle threads), then a
// smaller largest radix (smaller codelets)
constexpr bool better(const Plan &a, const Plan &c, int n) {
    if (c.k == 0) return true;
    if (a.k != c.k) return a.k < c.k;
    const int ba = bfly_per_thread(n, rmin_of(a)), bc = bfly_per_thread(n, rmin_of(c));
    if (ba != bc) return ba < bc;
    if (rmin_of(a) != rmin_of(c)) return rmin_of(a) > rmin_of(c);
    return rmax_of(a) < rmax_of(c);
}
constexpr void search(int n, int left, int from, Plan &cur, Plan &best) {
    if (left == 1) {
        if (better(cur, best, n)) best = cur;
        return;
    }
    if (cur.k == kMaxStages || (best.k != 0 && cur.k + 1 > best.k)) return;
    for (int i = from; i < kNumRadices; ++i) {
        if (left % kRadices[i]) continue;
        cur.r[cur.k++] = kRadices[i];
        search(n, left / kRadices[i], i, cur, best);
        --cur.k;
    }
}

constexpr Plan mixed_plan(int n) {
    Plan cur{}, p{};
    search(n, n, 0, cur, p);
    const int rmin = rmin_of(p), rmax0 = rmax_of(p);
    if (rmax0 >= 2 * rmin && n / rmax0 <= kMaxThreads) {
        // radices at least a factor two apart: one butterfly a thread in the
        // largest-radix stage and several in the smaller-radix ones, rather
        // than idle threads in the large one (measured faster at n = 375,
        // 2000 and 3000; slower at 1620 and 6000, whose radices are closer)
        p.t = n / rmax0;
        p.b = (n / rmin + p.t - 1) / p.t;
    } else {
        p.b = bfly_per_thread(n, rmin);
        p.t = (n / rmin + p.b - 1) / p.b;
    }
    p.vmax = 0;
    for (int s = 0; s < p.k; ++s) {
        const int bs = (n / p.r[s] + p.t - 1) / p.t;
        p.vmax = bs * p.r[s] > p.vmax ? bs * p.r[s] : p.vmax;
    }
    // Block shape and register budget.  The budget is at least what the
    // values held across a barrier need (two registers each, plus room for
    // indices, addresses and the codelets' temporaries; 48 for the 12- to
    // 16-point codelets, which need them to keep their loads in flight).
    // Blocks of at most 256 threads where a signal allows: many small blocks, so that one block's barriers stall few
    // threads and the blocks of an SM drift apart, some loading while others
    // compute.  Among the shapes that keep at least 1280 threads (40 warps)
    // of an SM busy, the largest budget (fewer registers cost loads in
    // flight), then the most busy threads, then the fewest signals a block;
    // if no shape reaches that, the most busy threads.
    const int rmax = rmax_of(p);
    int lower = 2 * p.vmax + 12;
    if (lower < 32) lower = 32;
    if (rmax >= 12 && lower < 48) lower = 48;
    const int sm1 = p.k > 1 ? n * 8 : 0;
    auto blocks_per_sm = [&](int threads, int smem, int regs) {
        int blocks = 2048 / threads;
        const int by_regs = 65536 / (threads * ((regs + 7) / 8 * 8));
        if (by_regs < blocks) blocks = by_regs;
        if (smem > 0 && kSmemPerSm / (smem + 1024) < blocks) blocks = kSmemPerSm / (smem + 1024);
        if (blocks > 32) blocks = 32;
        return blocks < 1 ? 1 : blocks;
    };
    constexpr int kBusyTarget = 1280;
    int best_ok = -1, best_regs = 0, best_busy = -1;
    const int max_spb = p.t >= 256 ? 1 : 256 / p.t;
    for (int spb = 1; spb <= max_spb; ++spb) {
        const int threads = (spb * p.t + 31) / 32 * 32;
        if (spb * sm1 > kSmemPerBlock) break;
        // budgets of 64, 56, 48 or 32 registers (at 40 the compiler spilled
        // the 10 x 10 x 10 kernel, slowing it by a fifth)
        for (int regs = 64; regs >= lower || regs == 64; regs -= (regs == 48 ? 16 : 8)) {
            const int r = regs > lower ? regs : lower;
            const int blocks = blocks_per_sm(threads, spb * sm1, r);
            const int busy = blocks * spb * p.t;
            const int ok = busy >= kBusyTarget ? 1 : 0;
            const bool take = ok != best_ok ? ok > best_ok
                              : ok ? (r != best_regs ? r > best_regs : busy > best_busy)
                                   : (busy != best_busy ? busy > best_busy : r > best_regs);
            if (take) {
                best_ok = ok;
                best_regs = r;
                best_busy = busy;
                p.spb = spb;
                p.threads = threads;
                p.minb = blocks;
            }
            if (regs <= lower) break;
        }
    }
    auto blocks_at = [&](int smem) { return blocks_per_sm(p.threads, smem, best_regs); };
    // a second buffer when it costs no block per SM
    p.dbl = p.k > 2 && 2 * p.spb * sm1 <= kSmemPerBlock && blocks_at(2 * p.spb * sm1) >= p.minb;
    return p;
}

constexpr int stage_len_before(const Plan &p, int s) {
    int l = 1;
    for (int i = 0; i < s; ++i) l *= p.r[i];
    return l;
}

// ---------------------------------------------------------------- kernel

// Stage S: the thread's butterflies b = t + i T (i < B_S), inputs read
// (from global memory in the first stage, else from the shared buffer),
// twiddled and transformed into v[i R + q].
template <int N, int S, int DIR>
__device__ __forceinline__ void stage_in(const float2 *src, const float2 *__restrict__ tw, int t, bool act, bool live,
                                         float2 *v) {
    constexpr Plan P = mixed_plan(N);
    constexpr int R = P.r[S], L = stage_len_before(P, S), m = N / (L * R), nb = N / R;
    constexpr int BS = (nb + P.t - 1) / P.t;
#pragma unroll
    for (int i = 0; i < BS; ++i) {
        const int b = t + i * P.t;
        if (!act || (nb % P.t != 0 && b >= nb)) continue;
        const int j = b / m, k = b - j * m;
        float2 u[R];
#pragma unroll
        for (int p = 0; p < R; ++p) {
            const int e = R * j * m + k + p * m;
            if constexpr (S == 0)
                u[p] = live ? __ldcs(src + e) : make_float2(0.f, 0.f);
            else
                u[p] = src[e];
        }
        if constexpr (S > 0) {
#pragma unroll
            for (int p = 1; p < R; ++p) {
                float2 w = __ldg(tw + p * j * m);  // W_n^(p j m) of the table exp(-2 pi i e / n)
                if (DIR > 0) w.y = -w.y;
                u[p] = cmul(u[p], w);
            }
        }
        dft_any<R, DIR>(u);
#pragma unroll
        for (int q = 0; q < R; ++q) v[i * R + q] = u[q];
    }
}

// Stage S's outputs to the shared buffer, or (LAST) to global memory
template <int N, int S, bool LAST>
__device__ __forceinline__ void stage_out(float2 *dst, int t, bool act, bool live, const float2 *v) {
    constexpr Plan P = mixed_plan(N);
    constexpr int R = P.r[S], L = stage_len_before(P, S), m = N / (L * R), nb = N / R, lm = L * m;
    constexpr int BS = (nb + P.t - 1) / P.t;
#pragma unroll
    for (int i = 0; i < BS; ++i) {
        const int b = t + i * P.t;
        if (!act || (nb % P.t != 0 && b >= nb)) continue;
        const int j = b / m, k = b - j * m;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int e = j * m + k + q * lm;
            if constexpr (LAST) {
                if (live) __stcs(dst + e, v[i * R + q]);
            } else {
                dst[e] = v[i * R + q];
            }
        }
    }
}

// v holds stage S - 1's outputs; write them, then run stage S onwards.
// One buffer: written in place, so every read of a stage is done (a second
// barrier) before its writes.  Two buffers: stage S - 1 writes buffer
// (S - 1) & 1, which nobody reads again before the barrier after stage S's
// writes to the other one.
template <int N, int S, int DIR>
__device__ __forceinline__ void stages_from(float2 *buf, float2 *buf2, float2 *gout, const float2 *__restrict__ tw,
                                            int t, bool act, bool live, float2 *v) {
    constexpr Plan P = mixed_plan(N);
    if constexpr (S == P.k) {
        stage_out<N, S - 1, true>(gout, t, act, live, v);
    } else {
        float2 *cur = P.dbl && ((S - 1) & 1) ? buf2 : buf;
        stage_out<N, S - 1, false>(cur, t, act, live, v);
        __syncthreads();
        stage_in<N, S, DIR>(cur, tw, t, act, live, v);
        if constexpr (!P.dbl && S + 1 < P.k) __syncthreads();
        stages_from<N, S + 1, DIR>(buf, buf2, gout, tw, t, act, live, v);
    }
}

template <int N, int DIR>
__global__ void __launch_bounds__(mixed_plan(N).threads, mixed_plan(N).minb)
    fft_mixed_kernel(const float2 *__restrict__ in, float2 *__restrict__ out, const float2 *__restrict__ tw,
                     int64_t batch) {
    constexpr Plan P = mixed_plan(N);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int s = static_cast<int>(threadIdx.x) / P.t;
    const bool act = s < P.spb;  // threads past spb t (the last warp's tail) only join the barriers
    const int t = static_cast<int>(threadIdx.x) - s * P.t;
    const int64_t sig = static_cast<int64_t>(blockIdx.x) * P.spb + s;
    const bool live = act && sig < batch;
    float2 *buf = reinterpret_cast<float2 *>(smem_raw) + (act ? s : 0) * N;
    float2 *buf2 = buf + (P.dbl ? P.spb * N : 0);
    float2 v[P.vmax];
    stage_in<N, 0, DIR>(in + sig * N, tw, t, act, live, v);
    stages_from<N, 1, DIR>(buf, buf2, out + sig * N, tw, t, act, live, v);
}

// ---------------------------------------------------------------- lookup

constexpr int count_lengths() {
    int c = 0;
    for (int n = 3; n <= kMixedMaxLen; ++n) c += has_kernel(n) ? 1 : 0;
    return c;
}
constexpr int kNumLengths = count_lengths();
struct Lengths {
    int v[kNumLengths];
};
constexpr Lengths make_lengths() {
    Lengths l{};
    int c = 0;
    for (int n = 3; n <= kMixedMaxLen; ++n)
        if (has_kernel(n)) l.v[c++] = n;
    return l;
}
constexpr Lengths kLengths = make_lengths();

}  // namespace mixed_detail

struct MixedLaunch {
    const void *fn;
    int threads, spb, smem, stages;
    int radices[mixed_detail::kMaxStages];
};

namespace mixed_detail {

template <int N>
bool fill(int n, int dir, MixedLaunch *o) {
    if (n != N) return false;
    constexpr Plan P = mixed_plan(N);
    o->fn = dir < 0 ? reinterpret_cast<const void *>(&fft_mixed_kernel<N, -1>)
                    : reinterpret_cast<const void *>(&fft_mixed_kernel<N, 1>);
    o->threads = P.threads;
    o->spb = P.spb;
    o->smem = P.k > 1 ? (P.dbl ? 2 : 1) * P.spb * N * static_cast<int>(sizeof(float2)) : 0;  // one stage: none
    o->stages = P.k;
    for (int i = 0; i < kMaxStages; ++i) o->radices[i] = i < P.k ? P.r[i] : 0;
    return true;
}
template <int K, size_t... I>
bool shard_lookup(int n, int dir, MixedLaunch *o, std::index_sequence<I...>) {
    bool found = false;
    ((found = found || fill<kLengths.v[K + static_cast<int>(I) * kMixedShards]>(n, dir, o)), ...);
    return found;
}

}  // namespace mixed_detail

// The kernels of lengths kLengths.v[K], kLengths.v[K + kMixedShards], ...
// (one translation unit each, compiled in parallel)
template <int K>
bool mixed_shard(int n, int dir, MixedLaunch *o) {
    constexpr int cnt = (mixed_detail::kNumLengths - K + kMixedShards - 1) / kMixedShards;
    return mixed_detail::shard_lookup<K>(n, dir, o, std::make_index_sequence<cnt>{});
}

bool mixed_shard_0(int n, int dir, MixedLaunch *o);
bool mixed_shard_1(int n, int dir, MixedLaunch *o);
bool mixed_shard_2(int n, int dir, MixedLaunch *o);
bool mixed_shard_3(int n, int dir, MixedLaunch *o);
bool mixed_shard_4(int n, int dir, MixedLaunch *o);
bool mixed_shard_5(int n, int dir, MixedLaunch *o);
bool mixed_shard_6(int n, int dir, MixedLaunch *o);
bool mixed_shard_7(int n, int dir, MixedLaunch *o);

}  // namespace bplg
