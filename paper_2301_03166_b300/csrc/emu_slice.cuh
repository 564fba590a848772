// emu_slice.cuh -- the slice digits of one FP64 value for the FP64-accurate
// products on the BF16 tensor cores (Ozaki splitting; k_emu.cu, k_resid_emu.cu),
// with integer operations only.
//
// With E_max the largest biased exponent of the value's row (at least 1),
// x = a / 2^(E_max - 1022) has |x| < 1, and F = round(|x| 2^56) is written in
// balanced base 128 from the least significant digit up: digits d_7 .. d_1 in
// [-64, 63] with a carry into the next, d_0 in [0, 128], so that
// x ~ sign(a) sum_{p=0}^{7} d_p 2^(-7 (p + 1)).  Each signed digit is exact in
// BF16.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace abft {

constexpr int EMU_SLICES = 8;

// The BF16 pattern of a small integer v (|v| <= 128, exact in BF16): the bits
// 0x4B400000 + v are the float 1.5 2^23 + v, so subtracting 1.5 2^23 gives v
// exactly as a float, whose low 16 bits are zero (at most 8 significant bits);
// its upper half is the BF16 pattern.  One integer add, one FP32 add and a
// shift instead of two conversions.
__device__ __forceinline__ uint16_t small_int_bf16(int v) {
    const float f = __fsub_rn(__int_as_float(0x4B400000 + v), 12582912.0f);
    return (uint16_t)(__float_as_uint(f) >> 16);
}

// The eight BF16 slice values (bit patterns) of the value with bits b.
__device__ __forceinline__ void slice_digits(unsigned long long b, int emax, uint16_t (&out)[8]) {
    const int e = (int)((b >> 52) & 0x7ffull);
    const unsigned long long mant = (b & 0xfffffffffffffull) | (e ? (1ull << 52) : 0ull);
    // F = round(mant 2^(E - E_max + 3)), E of a subnormal taken as 1: a right
    // shift by E_max - 3 - E (a left shift for the largest elements)
    const int sh = emax - 3 - (e ? e : 1);
    unsigned long long F;
    if (sh <= 0) F = mant << (-sh);
    else if (sh >= 64) F = 0ull;
    else F = (mant >> sh) + ((mant >> (sh - 1)) & 1ull);
    const bool neg = (b >> 63) != 0ull;
    int carry = 0;
#pragma unroll
    for (int p = EMU_SLICES - 1; p >= 0; --p) {
        int d = (int)((F >> (7 * (EMU_SLICES - 1 - p))) & 127ull) + carry;
        carry = 0;
        if (p > 0 && d >= 64) {
            d -= 128;
            carry = 1;
        }
        out[p] = small_int_bf16(neg ? -d : d);
    }
}

}  // namespace abft
