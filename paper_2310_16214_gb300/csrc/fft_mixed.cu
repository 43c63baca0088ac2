// Mixed-radix Stockham FFT for lengths n = 2^a 3^b 5^c that are not powers
// of two, the whole signal in shared memory.  (The paper keeps to N = r^n;
// this extends the radix-r Stockham formulation of Section III to products
// of small radices, so such lengths need not go through Bluestein's
// identity.)
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
// written out, the composite ones as two factors with their inner
// twiddles computed at compile time (float64 series, rounded once).  The
// factorisation takes the fewest stages; the block shape and the choice
// among such factorisations follow mixed_factor below.  Blocks hold nsig
// consecutive signals in two shared-memory buffers that the stages
// alternate between; the first stage reads global memory and the last
// writes it.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fft_common.cuh"
#include "internal.h"

namespace bplg {

namespace {

constexpr int kMixedMaxStages = 20;
constexpr int kMixedMaxThreads = 512;

// The stage radices, 4 bits a stage (an index into kRadices), first stage
// lowest; threads per signal (every stage's butterfly count is a multiple
// of it) and signals per block.
constexpr int kNumRadices = 11;
constexpr int kRadices[kNumRadices] = {16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};
struct MixedPlan {
    int nst;
    uint64_t codes;
    int r[kMixedMaxStages];  // host side
    int nsig, threads;
};
__host__ __device__ __forceinline__ int radix_of_code(uint64_t codes, int s) {
    switch (static_cast<int>((codes >> (4 * s)) & 15u)) {
        case 0: return 16;
        case 1: return 15;
        case 2: return 12;
        case 3: return 10;
        case 4: return 9;
        case 5: return 8;
        case 6: return 6;
        case 7: return 5;
        case 8: return 4;
        case 9: return 3;
        default: return 2;
    }
}

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

// Per-stage constants, computed once per block into shared memory: m (the
// stage's m'), L m (the output stride), and the multipliers that turn the
// divisions by m and by n / r into one high multiply: for 0 <= x, d < 2^14
// and M = floor((2^32 - 1) / d) + 1, floor(x / d) = (x M) >> 32 (M exceeds
// 2^32 / d by less than 1, and x (M - 2^32 / d) / 2^32 < 1 / d).  A divisor
// of 1 keeps x.
struct StageC {
    int m, lm, nb;
    uint32_t mm, mnb;
};
__device__ __forceinline__ uint32_t div_magic(int d) { return d > 1 ? 0xFFFFFFFFu / static_cast<uint32_t>(d) + 1u : 0u; }
__device__ __forceinline__ int udiv(int x, int d, uint32_t magic) {
    return d > 1 ? static_cast<int>(__umulhi(static_cast<uint32_t>(x), magic)) : x;
}

// One radix-R stage over the block's nsig signals.  FIRST: the inputs come
// from global memory (rows of signals sig0 .. sig0 + nvalid - 1, zeros past
// them); LAST: the outputs go to global memory (valid rows only).
// Otherwise src and dst are the shared-memory buffers.
template <int R, int DIR, bool FIRST, bool LAST>
__device__ __forceinline__ void mixed_stage(const float2 *src, float2 *dst, const float2 *__restrict__ tw, int n,
                                            const StageC &c, int nsig, int nvalid) {
    const int m = c.m, nb = c.nb, lm = c.lm;
    for (int b = threadIdx.x; b < nb * nsig; b += blockDim.x) {
        const int sig = nsig == 1 ? 0 : udiv(b, nb, c.mnb);
        const int bb = b - sig * nb;
        const int j = FIRST ? 0 : (LAST ? bb : udiv(bb, m, c.mm));
        const int jm = j * m;
        const int k = bb - jm;
        const bool live = sig < nvalid;
        const float2 *s = src + sig * n + R * jm + k;
        float2 v[R];
#pragma unroll
        for (int p = 0; p < R; ++p) {
            if (FIRST)
                v[p] = live ? __ldcs(s + p * m) : make_float2(0.f, 0.f);
            else
                v[p] = s[p * m];
        }
        if (!FIRST && j > 0) {
#pragma unroll
            for (int p = 1; p < R; ++p) {
                float2 w = __ldg(tw + p * jm);  // W_n^(p j m) of the table exp(-2 pi i e / n)
                if (DIR > 0) w.y = -w.y;
                v[p] = cmul(v[p], w);
            }
        }
        dft_any<R, DIR>(v);
        float2 *d = dst + sig * n + jm + k;
        if (LAST) {
            if (live) {
#pragma unroll
                for (int q = 0; q < R; ++q) __stcs(d + q * lm, v[q]);
            }
        } else {
#pragma unroll
            for (int q = 0; q < R; ++q) d[q * lm] = v[q];
        }
    }
}

template <int DIR, bool FIRST, bool LAST>
__device__ __forceinline__ void mixed_stage_r(int r, const float2 *src, float2 *dst, const float2 *__restrict__ tw,
                                              int n, const StageC &c, int nsig, int nvalid) {
    switch (r) {
        case 2: mixed_stage<2, DIR, FIRST, LAST>(src, dst, tw, n, c, nsig, nvalid); break;
        case 3: mixed_stage<3, DIR, FIRST, LAST>(src, dst, tw, n, c, nsig, nvalid); break;
        case 4: mixed_stage<4, DIR, FIRST, LAST>(src, dst, tw, n, c, nsig, nvalid); break;
        case 5: mixed_stage<5, DIR, FIRST, LAST>(src, dst, tw, n, c, nsig, nvalid); break;
        case 6: mixed_stage<6, DIR, FIRST, LAST>(src, dst, tw, n, c, nsig, nvalid); break;
        case 8: mixed_stage<8, DIR, FIRST, LAST>(src, dst, tw, n, c, nsig, nvalid); break;
        case 9: mixed_stage<9, DIR, FIRST, LAST>(src, dst, tw, n, c, nsig, nvalid); break;
        case 10: mixed_stage<10, DIR, FIRST, LAST>(src, dst, tw, n, c, nsig, nvalid); break;
        case 12: mixed_stage<12, DIR, FIRST, LAST>(src, dst, tw, n, c, nsig, nvalid); break;
        case 15: mixed_stage<15, DIR, FIRST, LAST>(src, dst, tw, n, c, nsig, nvalid); break;
        default: mixed_stage<16, DIR, FIRST, LAST>(src, dst, tw, n, c, nsig, nvalid); break;
    }
}

// The first stage reads the block's signals from global memory and the last
// writes them back; the stages between alternate between two shared-memory
// buffers.
template <int DIR>
__global__ void __launch_bounds__(kMixedMaxThreads, 2)
    fft_mixed_kernel(const float2 *__restrict__ in, float2 *__restrict__ out, const float2 *__restrict__ tw,
                     int nst, uint64_t codes, int n, int nsig, int64_t batch) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ StageC sc[kMixedMaxStages];
    __shared__ int sr[kMixedMaxStages];
    float2 *buf0 = reinterpret_cast<float2 *>(smem_raw), *buf1 = buf0 + nsig * n;
    const int64_t sig0 = static_cast<int64_t>(blockIdx.x) * nsig;
    const int64_t left = batch - sig0;
    const int nvalid = static_cast<int>(left < nsig ? left : nsig);
    const float2 *gin = in + sig0 * n;
    float2 *gout = out + sig0 * n;
    if (threadIdx.x < nst) {
        const int s = threadIdx.x;
        int L = 1;
        for (int i = 0; i < s; ++i) L *= radix_of_code(codes, i);
        const int r = radix_of_code(codes, s);
        StageC c;
        c.m = n / (L * r);
        c.lm = L * c.m;
        c.nb = n / r;
        c.mm = div_magic(c.m);
        c.mnb = div_magic(c.nb);
        sc[s] = c;
        sr[s] = r;
    }
    __syncthreads();
    if (nst == 1) {  // n = 3 or 5
        mixed_stage_r<DIR, true, true>(sr[0], gin, gout, tw, n, sc[0], nsig, nvalid);
        return;
    }
    mixed_stage_r<DIR, true, false>(sr[0], gin, buf0, tw, n, sc[0], nsig, nvalid);
    __syncthreads();
    for (int s = 1; s < nst - 1; ++s) {
        const float2 *src = (s & 1) ? buf0 : buf1;
        float2 *dst = (s & 1) ? buf1 : buf0;
        mixed_stage_r<DIR, false, false>(sr[s], src, dst, tw, n, sc[s], nsig, nvalid);
        __syncthreads();
    }
    const int last = nst - 1;
    mixed_stage_r<DIR, false, true>(sr[last], (last & 1) ? buf0 : buf1, gout, tw, n, sc[last], nsig, nvalid);
}

// The stage radices of n (false unless n = 2^a 3^b 5^c) and the block
// shape.  Blocks hold nsig signals (several below 512 points, within 24 KB
// of shared memory) and T threads, T = the largest stage's butterfly count
// rounded up to whole warps (at most kMixedMaxThreads), so no stage waits on
// a second pass of a few threads when one pass could do; among the
// factorisations with the fewest stages the one with the fewest passes
// (sum over stages of ceil(butterflies / T)) is taken, then the one with
// the largest smallest radix.
void mixed_search(int64_t left, int depth, int *cur, int *best_len, std::vector<std::vector<int>> *found) {
    if (left == 1) {
        if (depth < *best_len) {
            *best_len = depth;
            found->clear();
        }
        if (depth == *best_len) found->push_back(std::vector<int>(cur, cur + depth));
        return;
    }
    if (depth + 1 > *best_len || depth >= kMixedMaxStages) return;
    for (int i = 0; i < kNumRadices; ++i) {
        const int r = kRadices[i];
        if (left % r) continue;
        if (depth > 0 && r > cur[depth - 1]) continue;  // non-increasing: each multiset once
        cur[depth] = r;
        mixed_search(left / r, depth + 1, cur, best_len, found);
    }
}

bool mixed_factor(int64_t n, MixedPlan *mp) {
    int64_t v = n;
    while (v % 2 == 0) v /= 2;
    while (v % 3 == 0) v /= 3;
    while (v % 5 == 0) v /= 5;
    if (v != 1 || n < 3) return false;
    int cur[kMixedMaxStages];
    int best_len = kMixedMaxStages + 1;
    std::vector<std::vector<int>> found;
    mixed_search(n, 0, cur, &best_len, &found);
    if (found.empty() || best_len > 16) return false;
    const int64_t nsig = n >= 512 ? 1 : std::min<int64_t>(64, std::max<int64_t>(1, 1536 / n));
    int64_t best_passes = -1, best_t = 0;
    int best_min = 0;
    const std::vector<int> *pick = nullptr;
    for (const auto &f : found) {
        int64_t most = 0;
        int rmin = 16;
        for (int r : f) {
            most = std::max<int64_t>(most, nsig * (n / r));
            rmin = std::min(rmin, r);
        }
        const int64_t t = std::min<int64_t>(kMixedMaxThreads, (most + 31) / 32 * 32);
        int64_t passes = 0;
        for (int r : f) passes += (nsig * (n / r) + t - 1) / t;
        if (!pick || passes < best_passes || (passes == best_passes && rmin > best_min)) {
            pick = &f;
            best_passes = passes;
            best_t = t;
            best_min = rmin;
        }
    }
    mp->nst = best_len;
    mp->codes = 0;
    for (int i = 0; i < best_len; ++i) {
        mp->r[i] = (*pick)[i];
        int c = 0;
        while (kRadices[c] != mp->r[i]) ++c;
        mp->codes |= static_cast<uint64_t>(c) << (4 * i);
    }
    mp->nsig = static_cast<int>(nsig);
    mp->threads = static_cast<int>(best_t);
    return true;
}

std::mutex g_mu;
std::map<std::pair<int, int64_t>, float2 *> g_tables;  // (device, n) -> exp(-2 pi i e / n), e < n

int table_for(int64_t n, const float2 **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_tables.find(std::make_pair(dev, n));
    if (it != g_tables.end()) {
        *out = it->second;
        return BPLG_OK;
    }
    std::vector<float2> h(static_cast<size_t>(n));
    for (int64_t k = 0; k < n; ++k) {
        const double ang = -2.0 * M_PI * static_cast<double>(k) / static_cast<double>(n);
        h[static_cast<size_t>(k)] = make_float2(static_cast<float>(std::cos(ang)), static_cast<float>(std::sin(ang)));
    }
    float2 *d = nullptr;
    if ((e = cudaMalloc(&d, static_cast<size_t>(n) * sizeof(float2))) != cudaSuccess)
        return cuda_error(e, "mixed-radix twiddles");
    if ((e = cudaMemcpy(d, h.data(), static_cast<size_t>(n) * sizeof(float2), cudaMemcpyHostToDevice)) !=
        cudaSuccess) {
        cudaFree(d);
        return cuda_error(e, "mixed-radix twiddles upload");
    }
    g_tables[std::make_pair(dev, n)] = d;
    *out = d;
    return BPLG_OK;
}

}  // namespace

bool fft_mixed_supported(int64_t n) {
    MixedPlan mp;
    return n > 2 && n <= kMixedMaxN && !is_pow2(n) && mixed_factor(n, &mp);
}

int fft_mixed_launch(const void *in, void *out, int64_t n, int64_t batch, int dir, cudaStream_t s) {
    MixedPlan mp;
    if (!fft_mixed_supported(n) || !mixed_factor(n, &mp))
        return set_error(BPLG_ERR_UNSUPPORTED_SIZE, "fft (mixed radix): n must be 2^a 3^b 5^c, not a power of two, "
                                                    "at most " + std::to_string(kMixedMaxN));
    const float2 *tw = nullptr;
    int rc = table_for(n, &tw);
    if (rc != BPLG_OK) return rc;
    const int nsig = mp.nsig;
    const int64_t elems = nsig * n;
    const int threads = mp.threads;
    const int smem = static_cast<int>(2 * elems * static_cast<int64_t>(sizeof(float2)));
    const void *f = dir < 0 ? reinterpret_cast<const void *>(&fft_mixed_kernel<-1>)
                            : reinterpret_cast<const void *>(&fft_mixed_kernel<1>);
    rc = ensure_smem_attr(f, smem);
    if (rc != BPLG_OK) return rc;
    const int64_t blocks = (batch + nsig - 1) / nsig;
    rc = check_grid(blocks, "fft (mixed radix)");
    if (rc != BPLG_OK) return rc;
    const float2 *xi = static_cast<const float2 *>(in);
    float2 *xo = static_cast<float2 *>(out);
    int ni = static_cast<int>(n);
    int nsg = nsig;
    int nst = mp.nst;
    uint64_t codes = mp.codes;
    void *args[] = {(void *)&xi, (void *)&xo, (void *)&tw, &nst, &codes, &ni, &nsg, &batch};
    cudaError_t e = cudaLaunchKernel(f, dim3(static_cast<unsigned>(blocks)), dim3(threads), args,
                                     static_cast<size_t>(smem), s);
    return e == cudaSuccess ? BPLG_OK : launch_error(e, "fft (mixed radix) launch", f, blocks, threads, smem);
}

}  // namespace bplg
