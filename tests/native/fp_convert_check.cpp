// Host check of the integer float<->double conversions against the host's own
// IEEE-754 conversions (round to nearest even): bit-for-bit, NaN for NaN.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "fp_convert.cuh"

static uint64_t bits64(double d) { uint64_t v; std::memcpy(&v, &d, 8); return v; }
static double from64(uint64_t v) { double d; std::memcpy(&d, &v, 8); return d; }
static uint32_t bits32(float f) { uint32_t v; std::memcpy(&v, &f, 4); return v; }
static float from32(uint32_t v) { float f; std::memcpy(&f, &v, 4); return f; }

static uint64_t state = 0x243F6A8885A308D3ull;
static uint64_t next() {  // xorshift64*
    state ^= state >> 12; state ^= state << 25; state ^= state >> 27;
    return state * 0x2545F4914F6CDD1Dull;
}

static long fails = 0;
static void widen_case(uint32_t u, int k) {
    const float f = from32(u);
    const double got = fpc::widen_f32_pow2(f, k);
    const double ref = std::ldexp(static_cast<double>(f), k);
    if (std::isnan(ref) ? !std::isnan(got) : bits64(got) != bits64(ref)) {
        if (fails++ < 10) std::printf("widen %08x k=%d: got %016llx want %016llx\n", u, k,
                                      (unsigned long long)bits64(got), (unsigned long long)bits64(ref));
    }
    // the zero-or-normal form, and the predicate that selects it
    const bool zn = f == 0.0f || std::isnormal(f);
    if (fpc::f32_zero_or_normal(f) != zn) {
        if (fails++ < 10) std::printf("zero_or_normal %08x: got %d\n", u, int(!zn));
    }
    if (zn && k == 0 && bits64(fpc::widen_f32_normal(f)) != bits64(static_cast<double>(f))) {
        if (fails++ < 10) std::printf("widen_normal %08x\n", u);
    }
}
static void narrow_case(uint64_t v) {
    const double x = from64(v);
    const float ref = static_cast<float>(x);
    const float got = fpc::narrow_f64(x);
    if (std::isnan(ref) ? !std::isnan(got) : bits32(got) != bits32(ref)) {
        if (fails++ < 10) std::printf("narrow %016llx: got %08x want %08x\n", (unsigned long long)v, bits32(got), bits32(ref));
    }
    // flush-to-zero variant: inputs below 2^-126 in magnitude give a signed zero
    const float ref_ftz = std::fabs(x) < std::ldexp(1.0, -126) ? std::copysign(0.0f, static_cast<float>(x)) : ref;
    const float got_ftz = fpc::narrow_f64_ftz(x);
    if (std::isnan(ref_ftz) ? !std::isnan(got_ftz) : bits32(got_ftz) != bits32(ref_ftz)) {
        if (fails++ < 10) std::printf("narrow_ftz %016llx: got %08x want %08x\n", (unsigned long long)v, bits32(got_ftz), bits32(ref_ftz));
    }
}

// scaled narrowing: (x * 2^k) rounded to float with flush to zero below
// 2^-126, for doubles x that are zero or normal (x * 2^k computed exactly by
// ldexp: the tested k keep it normal in float64)
static void narrow_pow2_case(uint64_t v, int k) {
    const double x = from64(v);
    if (std::fpclassify(x) == FP_SUBNORMAL) return;
    const double xs = std::ldexp(x, k);
    const float ref = std::fabs(xs) < std::ldexp(1.0, -126) ? std::copysign(0.0f, static_cast<float>(xs))
                                                             : static_cast<float>(xs);
    const float got = fpc::narrow_f64_ftz_pow2(x, k);
    if (std::isnan(ref) ? !std::isnan(got) : bits32(got) != bits32(ref)) {
        if (fails++ < 10) std::printf("narrow_pow2 %016llx k=%d: got %08x want %08x\n", (unsigned long long)v, k,
                                      bits32(got), bits32(ref));
    }
}

int main() {
    long n_w = 0, n_n = 0;
    // widen: every 61st bit pattern, all subnormals near the ends, all specials
    for (uint64_t u = 0; u <= 0xFFFFFFFFull; u += 61, ++n_w) widen_case(static_cast<uint32_t>(u), 0);
    for (uint32_t u = 0; u < 0x00100000u; ++u, n_w += 2) { widen_case(u, 0); widen_case(u | 0x80000000u, 0); }
    for (uint32_t u = 0x007F0000u; u < 0x00810000u; ++u, ++n_w) widen_case(u, 0);
    for (uint32_t u = 0x7F7F0000u; u <= 0x7FFFFFFFu && u >= 0x7F7F0000u; ++u, n_w += 2) { widen_case(u, 0); widen_case(u | 0x80000000u, 0); }
    for (int k = -700; k <= 700; k += 7)
        for (int j = 0; j < 20000; ++j, ++n_w) widen_case(static_cast<uint32_t>(next()), k);
    // narrow: random patterns over the whole range
    for (int j = 0; j < 40000000; ++j, ++n_n) narrow_case(next());
    // narrow: doubles whose exponent lies in or near the float range
    for (int j = 0; j < 40000000; ++j, ++n_n) {
        const uint64_t r = next();
        const uint64_t e = 896 - 30 + (r >> 55) % 300;  // biased double exponents 866..1165
        narrow_case((r & 0x800FFFFFFFFFFFFFull) | (e << 52));
    }
    // narrow: exact float midpoints and their double neighbours, normal and subnormal
    for (int j = 0; j < 20000000; ++j) {
        uint32_t u = static_cast<uint32_t>(next());
        if ((u & 0x7F800000u) == 0x7F800000u) continue;
        const double lo = static_cast<double>(from32(u));
        const uint32_t un = u + 1;
        const double hi = ((un & 0x7F800000u) == 0x7F800000u) ? std::ldexp(1.0, 128) * (u >> 31 ? -1 : 1)
                                                                  : static_cast<double>(from32(un));
        const double mid = 0.5 * (lo + hi);  // exact: both are floats, sum fits in 53 bits
        const uint64_t m = bits64(mid);
        narrow_case(m); narrow_case(m + 1); narrow_case(m - 1);
        n_n += 3;
    }
    // narrow: the overflow edge and the underflow edge, including zeros and specials
    const double edges[] = {0.0, -0.0, 3.4028234663852886e38, 3.4028235677973366e38, 3.4028235677973362e38,
                            std::ldexp(1.0, 128), 1e300, -1e300, INFINITY, -INFINITY, NAN,
                            std::ldexp(1.0, -149), std::ldexp(1.0, -150), std::ldexp(1.5, -150), std::ldexp(1.0, -151),
                            std::ldexp(1.0, -126), std::ldexp(0.99999999, -126), 5e-324, 1e-310};
    for (double x : edges) { narrow_case(bits64(x)); narrow_case(bits64(-x)); n_n += 2; }
    // scaled narrowing: exponents around the float range, shifts up to +-300
    for (int j = 0; j < 20000000; ++j, ++n_n) {
        const uint64_t r = next();
        const int k = static_cast<int>((r >> 40) % 601) - 300;
        const uint64_t e = static_cast<uint64_t>(896 - 40 - k + static_cast<int>((r >> 52) % 340));
        if (e < 1 || e > 2046) continue;
        narrow_pow2_case((r & 0x800FFFFFFFFFFFFFull) | (e << 52), k);
    }
    for (int k = -300; k <= 300; ++k) {
        for (double x : edges) { narrow_pow2_case(bits64(x), k); narrow_pow2_case(bits64(-x), k); }
        narrow_pow2_case(bits64(std::ldexp(1.0, -126 - k)), k);
        narrow_pow2_case(bits64(std::ldexp(0.75, -126 - k)), k);
        n_n += 2 * 19 + 2;
    }
    std::printf("%s widen=%ld narrow=%ld fails=%ld\n", fails ? "FAIL" : "OK", n_w, n_n, fails);
    return fails ? 1 : 0;
}
