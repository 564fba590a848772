// fp_bits.cuh -- conversions built from the IEEE-754 binary64 / binary32
// definitions with integer operations only.  B300 issues every FP64 instruction, conversions
// included, at about one warp instruction per 64 clocks per sub-partition, so
// epilogues that would otherwise convert on the FP64 pipe assemble the bits
// themselves.
#pragma once

#include <stdint.h>

namespace abft {

// acc * 2^s rounded to nearest (ties to even), as a double: the magnitude is
// normalized with a count of leading zeros, its top 53 bits are rounded on the
// 11 bits below them, and s is folded into the exponent field.  ok = false
// when the result would be subnormal or overflow (the caller converts on the
// FP64 pipe).
__device__ __forceinline__ double i64_scaled_to_f64(long long acc, int s, bool& ok) {
    ok = true;
    if (acc == 0) return 0.0;
    const unsigned long long sign = acc < 0 ? 0x8000000000000000ull : 0ull;
    unsigned long long u = acc < 0 ? 0ull - (unsigned long long)acc : (unsigned long long)acc;
    const int lz = __clzll((long long)u);
    u <<= lz;                                          // leading one at bit 63
    unsigned long long mant = u >> 11;                 // 53 bits, leading one at bit 52
    const unsigned long long rem = u & 0x7ffull;
    if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) ++mant;
    int e = 1086 - lz + s;                             // biased exponent of mant 2^(11 - lz + s)
    if (mant >> 53) {                                  // rounding carried into bit 53
        mant >>= 1;
        ++e;
    }
    if (e <= 0 || e >= 2047) {
        ok = false;
        return 0.0;
    }
    return __longlong_as_double((long long)(sign | ((unsigned long long)e << 52) |
                                            (mant & 0xfffffffffffffull)));
}

// Exact float -> double with integer operations only: rebias the exponent and
// widen the mantissa; subnormals are normalized with a count of leading
// zeros; zero, infinities and NaN keep their class.
__device__ __forceinline__ double f32_to_f64_exact(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t sign = b & 0x80000000u, e = (b >> 23) & 0xffu;
    uint32_t m = b & 0x7fffffu, ed;
    if (e == 0xffu) {
        ed = 0x7ffu;
    } else if (e != 0u) {
        ed = e + 896u;                         // (e - 127) + 1023
    } else if (m == 0u) {
        ed = 0u;
    } else {                                   // m 2^-149, leading one at bit 31 - clz
        const uint32_t sh = (uint32_t)__clz((int)m) - 8u;
        m = (m << sh) & 0x7fffffu;
        ed = 897u - sh;                        // (-126 - sh) + 1023
    }
    const uint32_t hi = sign | (ed << 20) | (m >> 3);
    const uint32_t lo = m << 29;
    return __hiloint2double((int)hi, (int)lo);
}

// |x| as a float by integer operations, the mantissa truncated (for
// diagnostics such as ratios, where a relative error below 2^-23 does not
// matter): 0 below the float range, infinity above it and for Inf / NaN.
__device__ __forceinline__ float f64_abs_to_f32_trunc(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
    const int e = (int)(b >> 52);
    if (e >= 2047 || e > 1023 + 127) return __uint_as_float(0x7f800000u);
    if (e < 1023 - 126) return 0.0f;
    const uint32_t m = (uint32_t)((b >> 29) & 0x7fffffull);
    return __uint_as_float(((uint32_t)(e - 896) << 23) | m);
}

// x rounded to nearest (ties to even) in a 16-bit format with EB exponent bits
// and MB mantissa bits (BF16: 8, 7; FP16: 5, 10), as its bit pattern, by integer
// operations on the binary64 fields: normal results keep the top MB bits of the
// significand and round on the 52 - MB bits below; results below the format's
// normal range are multiples of its smallest subnormal 2^(1 - bias - MB),
// rounded the same way (a carry out of the subnormal range gives the smallest
// normal number, as the encoding implies).  ok = false for NaN, infinities and
// values that would overflow (the caller converts those on the FP64 pipe).
template <int EB, int MB>
__device__ __forceinline__ uint32_t f64_to_small_rn(double x, bool& ok) {
    constexpr int BIAS = (1 << (EB - 1)) - 1;
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t sgn = (uint32_t)(b >> 63) << (EB + MB);
    const int e = (int)((b >> 52) & 0x7ffull);
    ok = true;
    if (e == 0) return sgn;                        // zero, FP64 subnormal: below half an ulp
    if (e == 0x7ff) {
        ok = false;
        return 0u;
    }
    const int E = e - 1023;
    const unsigned long long full = (b & 0xfffffffffffffull) | (1ull << 52);
    int sh;                                        // bits dropped from the 53-bit significand
    uint32_t ebits;
    if (E >= 1 - BIAS) {                           // normal in the small format
        sh = 52 - MB;
        ebits = (uint32_t)(E + BIAS);
    } else {                                       // subnormal: units of 2^(1 - BIAS - MB)
        sh = 52 - MB + (1 - BIAS - E);
        ebits = 0u;
        if (sh > 54) return sgn;                   // below half the smallest subnormal
    }
    unsigned long long q = full >> sh;
    const unsigned long long rem = full & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (q & 1ull))) ++q;
    uint32_t r;
    if (ebits) {                                   // q in [2^MB, 2^(MB+1)]: hidden bit in q
        r = (ebits << MB) + (uint32_t)(q - (1ull << MB));
        if (r >= ((1u << EB) - 1u) << MB) {        // rounded up to infinity
            ok = false;
            return 0u;
        }
    } else {
        r = (uint32_t)q;                           // a carry to 2^MB is the smallest normal
    }
    return sgn | r;
}

// a >> s for any s; PTX clamps shift amounts above 31 to 32 (a result of 0)
__device__ __forceinline__ uint32_t shr_clamp(uint32_t a, uint32_t s) {
    uint32_t d;
    asm("shr.b32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(s));
    return d;
}

// An entry as a signed multiple of 2^(vexp - 1075), truncated toward zero (less
// than one unit off): its 53-bit significand shifted right by vexp - e in two
// 32-bit words (a funnel shift for the low word, clamped shifts for the rest),
// the sign applied as (q ^ s) - s.  emax collects the biased exponents e: an
// entry above the bound, or not finite, leaves emax > vexp, which the caller
// checks once per tile.  Zeros and subnormals (e = 0) are read with the
// implicit bit set, which is below one unit for vexp >= 64: callers take the
// fixed-point sums only for such bounds.
__device__ __forceinline__ long long to_fixed(double x, int vexp, int& emax) {
    const uint32_t lo = (uint32_t)__double2loint(x), hi = (uint32_t)__double2hiint(x);
    const int e = (int)((hi >> 20) & 0x7ffu);
    emax = e > emax ? e : emax;
    const uint32_t mh = (hi & 0xfffffu) | 0x100000u;
    const uint32_t sh = (uint32_t)(vexp - e);
    const uint32_t ql = sh < 32u ? __funnelshift_rc(lo, mh, sh) : shr_clamp(mh, sh - 32u);
    const uint32_t qh = shr_clamp(mh, sh);
    const long long q = (long long)(((unsigned long long)qh << 32) | ql);
    const long long sg = (long long)((int)hi >> 31);
    return (q ^ sg) - sg;
}

// Smallest bound exponent for which to_fixed reads zeros correctly.
constexpr int kFixedMinExp = 64;

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace abft
