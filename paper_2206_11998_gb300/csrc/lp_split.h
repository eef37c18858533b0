// lp_split.h -- the split of an FP64 value into two floats, h = RN(x) and
// l = RN(x - h) (round to nearest, ties to even), by integer operations on the
// bit pattern.
//
// On this GPU the FP64 units, which also execute every conversion between
// double and float, run at a small fraction of the FP32 rate; the plain form
// of the split (two conversions to float, one back, one FP64 subtraction) made
// the gather of the state FP64-bound.  Here h is x's 53-bit significand
// rounded to 24 bits, and x - h, exact in double, is the remainder below those
// 24 bits (negative when h rounded up): an integer of at most 28 bits times
// 2^(e - 52), which is rounded to 24 bits again for l.  Both results are the
// ones the plain form gives; the host test (tests/test_split_host.py) checks
// that bit for bit against the compiler's conversions.
//
// Also the floor of an FP64 value as an integer, from its bits (floor_clamped).
//
// Plain C++ so that the host test compiles it as well.
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define LP_SPLIT_FN __host__ __device__ __forceinline__
#else
#define LP_SPLIT_FN inline
#endif

namespace lp {

LP_SPLIT_FN uint64_t split_bits_of(double x)
{
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    memcpy(&b, &x, sizeof b);
    return b;
#endif
}

LP_SPLIT_FN float split_float_of(uint32_t b)
{
#if defined(__CUDA_ARCH__)
    return __uint_as_float(b);
#else
    float f;
    memcpy(&f, &b, sizeof f);
    return f;
#endif
}

LP_SPLIT_FN int split_clz(uint32_t v)   // v != 0
{
#if defined(__CUDA_ARCH__)
    return __clz(v);
#else
    return __builtin_clz(v);
#endif
}

// bits of the float RN(a 2^s) for an integer 0 < a < 2^30 whose rounded value
// is a normal float
LP_SPLIT_FN uint32_t split_scaled_bits(uint32_t a, int s)
{
    const int p = 31 - split_clz(a);         // a's leading bit
    uint32_t m;                              // a's significand rounded to 24 bits
    if (p <= 23) {
        m = a << (23 - p);
    } else {
        const int sh = p - 23;
        m = a >> sh;
        const uint32_t r = a & ((1u << sh) - 1u), half = 1u << (sh - 1);
        if (r > half || (r == half && (m & 1u))) ++m;
    }
    // m in [2^23, 2^24]: exponent field p + s + 127 holding m - 2^23, written as
    // one addition so that m = 2^24 carries into the exponent
    return ((uint32_t)(p + s + 126) << 23) + m;
}

// h = RN(x) and l = RN(x - h) as floats.  Returns false, with h and l
// untouched, outside the range handled here: nonzero |x| below 2^-74 (where l
// could be subnormal), |x| of 2^127 and above (where h could overflow), inf
// and NaN; the caller then takes the FP64 form.
LP_SPLIT_FN bool split_exact(double x, float& h, float& l)
{
    const uint64_t b = split_bits_of(x);
    const uint32_t sgn = (uint32_t)(b >> 63) << 31;
    if ((b << 1) == 0ull) {                  // +-0
        h = split_float_of(sgn);
        l = 0.0f;
        return true;
    }
    const int e = (int)((b >> 52) & 0x7ffu) - 1023;
    if (e < -74 || e > 126) return false;
    const uint64_t S = (b & 0xfffffffffffffull) | (1ull << 52);   // 53-bit significand
    const uint32_t top = (uint32_t)(S >> 29);                     // its first 24 bits
    const uint32_t rem = (uint32_t)S & 0x1fffffffu;               // the other 29
    const bool up = rem > 0x10000000u || (rem == 0x10000000u && (top & 1u) != 0u);
    h = split_float_of(sgn | ((((uint32_t)(e + 126)) << 23) + top + (up ? 1u : 0u)));
    // x - h in units of 2^(e - 52): the remainder, less one unit of h when h
    // rounded up; at most 2^28 in magnitude
    int32_t rr = up ? (int32_t)rem - (1 << 29) : (int32_t)rem;
    if (rr == 0) {                           // x == h: x - h is +0
        l = 0.0f;
        return true;
    }
    uint32_t lsgn = sgn;
    if (rr < 0) {
        rr = -rr;
        lsgn ^= 0x80000000u;
    }
    l = split_float_of(lsgn | split_scaled_bits((uint32_t)rr, e - 52));
    return true;
}

// floor(t) as an unsigned integer clamped to [0, qmax] (qmax < 2^32), from the
// bits of t: 0 for t < 1, negative t and NaN; qmax for t >= qmax and +inf
LP_SPLIT_FN uint32_t floor_clamped(double t, uint32_t qmax)
{
    const uint64_t b = split_bits_of(t);
    if (b >> 63) return 0u;                                   // negative, -0, NaN with the sign set
    const int E = (int)((b >> 52) & 0x7ffu);
    const uint64_t mant = b & 0xfffffffffffffull;
    if (E == 0x7ff) return mant ? 0u : qmax;                  // NaN, +inf
    const int e = E - 1023;
    if (e < 0) return 0u;                                     // t < 1 (zero and subnormals included)
    if (e >= 32) return qmax;
    const uint32_t q = (uint32_t)((mant | (1ull << 52)) >> (52 - e));
    return q < qmax ? q : qmax;
}

// RN(x) as a float, the first half of split_exact; false outside its range
LP_SPLIT_FN bool round_exact(double x, float& h)
{
    float l;
    return split_exact(x, h, l);
}

}  // namespace lp
