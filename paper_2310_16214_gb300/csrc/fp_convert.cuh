// float32 <-> float64 conversions done with integer operations.
//
// On GB300 a float<->double conversion is issued to the FP64 pipe, which
// retires 2 operations per clock per SM (1/64 of the FP32 rate).  In the
// refinement (FP32 solve, FP64 residual r = d - A x, FP64 update x += e) a
// straightforward build spends more FP64-pipe slots on conversions (widening
// a, b, c, d and the correction, narrowing r) than on the residual's
// arithmetic.  The functions below produce the same bits as the IEEE-754
// conversions, with integer and bit operations on the 32-bit halves of the
// double, so only the residual's fused multiply-adds and the update's add
// remain on the FP64 pipe.
//
//   widen_f32(f)           exact float -> double (every finite value, ±0, ±inf,
//                          NaN stays NaN)
//   widen_f32_normal(f)    the same for zero or normal f (fewer operations)
//   widen_f32_pow2(f, k)   exact f * 2^k as a double, for |k| <= 700
//   narrow_f64(x)          double -> float rounded to nearest, ties to even,
//                          with overflow to ±inf and gradual underflow
//   narrow_f64_ftz(x)      the same, inputs below 2^-126 flushed to ±0
//   narrow_f64_ftz_pow2(x, k)  x * 2^k narrowed as narrow_f64_ftz, |k| <= 300
//
// IEEE-754 binary32: 1 sign, 8 exponent (bias 127), 23 fraction bits;
// binary64: 1 sign, 11 exponent (bias 1023), 52 fraction bits.  A normal
// float's fraction is the top 23 of the double's 52, and the biased exponent
// moves by 1023 - 127 = 896.  Both sides are plain header code so the host
// tests can check them against the host's own conversions.
#pragma once

#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define BPLG_FPC __host__ __device__ __forceinline__
#else
#define BPLG_FPC inline
#endif

namespace fpc {

BPLG_FPC uint32_t bits_f32(float f) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
#endif
}

BPLG_FPC float f32_from_bits(uint32_t u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    std::memcpy(&f, &u, 4);
    return f;
#endif
}

BPLG_FPC double f64_from_halves(uint32_t hi, uint32_t lo) {
#ifdef __CUDA_ARCH__
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
#else
    const uint64_t v = (static_cast<uint64_t>(hi) << 32) | lo;
    double d;
    std::memcpy(&d, &v, 8);
    return d;
#endif
}

BPLG_FPC uint32_t hi_f64(double x) {
#ifdef __CUDA_ARCH__
    return static_cast<uint32_t>(__double2hiint(x));
#else
    uint64_t v;
    std::memcpy(&v, &x, 8);
    return static_cast<uint32_t>(v >> 32);
#endif
}

BPLG_FPC uint32_t lo_f64(double x) {
#ifdef __CUDA_ARCH__
    return static_cast<uint32_t>(__double2loint(x));
#else
    uint64_t v;
    std::memcpy(&v, &x, 8);
    return static_cast<uint32_t>(v);
#endif
}

// f * 2^k exactly, for |k| <= 700 (every finite float's image stays
// normal).  Branch-free: a subnormal f is first scaled into the normal range
// by 2^64 in float arithmetic (exact, the product needs no rounding) and k
// drops by 64; zero and inf/NaN are selected at the end.
BPLG_FPC double widen_f32_pow2(float f, int k) {
    const bool sub = (bits_f32(f) & 0x7F800000u) == 0u;
    const uint32_t u = bits_f32(f * (sub ? 18446744073709551616.0f : 1.0f));
    k -= sub ? 64 : 0;
    const uint32_t sign = u & 0x80000000u;
    const uint32_t a = u & 0x7FFFFFFFu;
    uint32_t hi = sign | ((a >> 3) + (static_cast<uint32_t>(896 + k) << 20));
    hi = a == 0u ? sign : hi;
    hi = a >= 0x7F800000u ? (sign | 0x7FF00000u | ((a & 0x007FFFFFu) >> 3)) : hi;  // inf, NaN
    return f64_from_halves(hi, u << 29);
}

BPLG_FPC double widen_f32(float f) { return widen_f32_pow2(f, 0); }

// widen_f32 for a float known to be zero or normal (no subnormal, inf or
// NaN): the exponent rebias and the zero case only.
BPLG_FPC double widen_f32_normal(float f) {
    const uint32_t u = bits_f32(f);
    const uint32_t a = u & 0x7FFFFFFFu;
    const uint32_t hi = (u & 0x80000000u) | (a ? (a >> 3) + (896u << 20) : 0u);
    return f64_from_halves(hi, u << 29);
}

// true when f is zero or normal (widen_f32_normal applies)
BPLG_FPC bool f32_zero_or_normal(float f) {
    const uint32_t e = bits_f32(f) & 0x7F800000u;
    return (bits_f32(f) & 0x7FFFFFFFu) == 0u || (e != 0u && e != 0x7F800000u);
}

// double -> float, round to nearest even.  The 52-bit fraction splits into
// the 23 kept bits and 29 dropped ones; the dropped part decides the
// rounding (above half: up; exactly half: to the even neighbour).  A carry
// out of the fraction increments the exponent, and out of exponent 254 it
// gives the encoding of infinity, as IEEE requires.
BPLG_FPC float narrow_f64(double x) {
    const uint32_t hi = hi_f64(x), lo = lo_f64(x);
    const uint32_t sign = hi & 0x80000000u;
    const uint32_t ah = hi & 0x7FFFFFFFu;
    const int e = static_cast<int>(ah >> 20);
    const int fe = e - 896;  // biased float exponent
    if (fe >= 1 && fe <= 254) {
        const uint32_t base = (static_cast<uint32_t>(fe) << 23) | ((ah & 0x000FFFFFu) << 3) | (lo >> 29);
        const uint32_t rest = lo & 0x1FFFFFFFu;
        const uint32_t inc = (rest > 0x10000000u || (rest == 0x10000000u && (base & 1u))) ? 1u : 0u;
        return f32_from_bits(sign | (base + inc));
    }
    if (e == 0x7FF) {  // inf or NaN
        const bool nan = (ah & 0x000FFFFFu) != 0u || lo != 0u;
        return f32_from_bits(sign | (nan ? 0x7FC00000u : 0x7F800000u));
    }
    if (fe > 254) return f32_from_bits(sign | 0x7F800000u);
    // fe <= 0: the result is subnormal or zero.  Significand with its
    // leading one: 53 bits; the float keeps the bits above 2^-149.
    const int s = 1 - fe;  // extra right shift beyond the 29 dropped bits
    if (s > 25 || e == 0) return f32_from_bits(sign);  // below half the smallest subnormal
    const uint64_t sig = (static_cast<uint64_t>((ah & 0x000FFFFFu) | 0x00100000u) << 32) | lo;
    const int drop = 29 + s;
    const uint64_t q = sig >> drop;
    const uint64_t rem = sig & ((uint64_t(1) << drop) - 1);
    const uint64_t half = uint64_t(1) << (drop - 1);
    const uint64_t inc = (rem > half || (rem == half && (q & 1u))) ? 1u : 0u;
    return f32_from_bits(sign | static_cast<uint32_t>(q + inc));
}

// (x * 2^k) as a float, round to nearest even, with results below 2^-126 in
// magnitude flushed to signed zero (the flush-to-zero convention of FP32
// arithmetic), for |k| <= 300.  The scale is an offset of the exponent
// field, so it is exact and costs nothing; an x that is zero or a float64
// subnormal gives signed zero.  Branch-free; used where the float only feeds
// an FP32 solve (a residual narrowed after it has been scaled so that its
// largest entry lies in [1/2, 1)).
BPLG_FPC float narrow_f64_ftz_pow2(double x, int k) {
    const uint32_t hi = hi_f64(x), lo = lo_f64(x);
    const uint32_t sign = hi & 0x80000000u;
    const uint32_t ah = hi & 0x7FFFFFFFu;
    const int e = static_cast<int>(ah >> 20);
    const int fe = e == 0 || e == 0x7FF ? (e == 0 ? 0 : 255) : e - 896 + k;
    const uint32_t base = (static_cast<uint32_t>(fe) << 23) + (((ah & 0x000FFFFFu) << 3) | (lo >> 29));
    const uint32_t rest = lo & 0x1FFFFFFFu;
    const uint32_t inc = (rest > 0x10000000u || (rest == 0x10000000u && (base & 1u))) ? 1u : 0u;
    uint32_t r = sign | (base + inc);
    r = fe <= 0 ? sign : r;
    const bool nan = ah > 0x7FF00000u || (ah == 0x7FF00000u && lo != 0u);
    r = fe >= 255 ? (sign | (nan ? 0x7FC00000u : 0x7F800000u)) : r;
    return f32_from_bits(r);
}

// double -> float, round to nearest even, with inputs below 2^-126 in
// magnitude flushed to signed zero.
BPLG_FPC float narrow_f64_ftz(double x) { return narrow_f64_ftz_pow2(x, 0); }

}  // namespace fpc
