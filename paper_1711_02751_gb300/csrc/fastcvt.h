// FP64 <-> FP32 conversions on the integer pipes.
//
// GB300 executes the F2F conversions between FP64 and FP32 at its FP64 rate -- measured 1.8
// results per clock per SM, the same as an FP64 add, against ~110 FP32 adds -- so a kernel that
// converts every element it loads or stores spends most of its time there rather than on HBM.
// These build the target's bit pattern with 32-bit integer shifts, adds and selects on the two
// words of the double instead (the exponent rebias 1023 - 127 = 896 and the 52 - 23 = 29 mantissa
// bits that separate the formats).
//
// f64_to_f32 rounds to nearest with ties away from zero (IEEE would break ties to even: the two
// differ only when the 29 dropped bits are exactly 1000...0).  Magnitudes below 2^-126 flush to a
// signed zero, at or above 2^128 they become infinities, and NaN stays NaN.  f32_to_f64 is exact
// for normal numbers and zero; FP32 subnormals flush to zero.
#pragma once

namespace hdgdg {

__device__ __forceinline__ float f64_to_f32(double v) {
    const unsigned hw = (unsigned)__double2hiint(v), lw = (unsigned)__double2loint(v);
    const unsigned sign = hw & 0x80000000u, mh = hw & 0x7FFFFFFFu;   // exponent (11) | top 20 mantissa bits
    const unsigned e11 = mh >> 20;
    // rebased exponent and top 23 mantissa bits, plus the rounding bit (carries into the exponent)
    unsigned f = (((mh - (896u << 20)) << 3) | (lw >> 29)) + ((lw >> 28) & 1u);
    f = e11 <= 896u ? 0u : f;
    f = e11 >= 1151u ? (e11 == 2047u && ((mh & 0xFFFFFu) | lw) != 0u ? 0x7FC00000u : 0x7F800000u) : f;
    return __uint_as_float(sign | f);
}

__device__ __forceinline__ double f32_to_f64(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned sign = u & 0x80000000u, mag = u & 0x7FFFFFFFu;
    const unsigned e8 = mag >> 23;
    unsigned hw = (mag >> 3) + (896u << 20);
    unsigned lw = mag << 29;
    hw = e8 == 0u ? 0u : hw;
    lw = e8 == 0u ? 0u : lw;
    hw = e8 == 255u ? (0x7FF00000u | ((mag >> 3) & 0xFFFFFu)) : hw;
    return __hiloint2double((int)(hw | sign), (int)lw);
}

// Storage-type helpers for kernels templated on their arithmetic type T (double or float).
template <typename T>
__device__ __forceinline__ T from_f64(double v) {
    if constexpr (sizeof(T) == 4) return f64_to_f32(v);
    else return v;
}

template <typename T>
__device__ __forceinline__ double to_f64(T v) {
    if constexpr (sizeof(T) == 4) return f32_to_f64(v);
    else return v;
}

}  // namespace hdgdg
