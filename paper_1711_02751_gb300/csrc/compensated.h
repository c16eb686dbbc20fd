// FP64-class sums on the FP32 pipes.  GB300 issues FP32 FMAs at 64x its FP64 rate, so FP64-bound
// contractions keep their operand as an unevaluated pair of FP32 arrays (a = a_hi + a_lo, the
// same 8 bytes per entry as FP64) and form each dot product with the compensated Dot2 of Ogita,
// Rump and Oishi (SIAM J. Sci. Comput. 26, 2005): the products a_hi x_hi are split exactly with
// Dekker's TwoProduct (via FMA) and summed with Knuth's TwoSum, and the cross terms
// a_hi x_lo + a_lo x_hi are added in FP32.  The result carries about 48 bits (~1e-13 relative,
// against 1e-16 for FP64 arithmetic) at the memory bound instead of the FP64 bound.  The
// explicit _rn intrinsics keep the compiler from fusing the steps.
#pragma once

#include "fastcvt.h"

namespace hdgdg {

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

struct Dot2 {
    float p = 0.f, c = 0.f;   // running sum and its accumulated correction
    __device__ __forceinline__ void add(float ah, float al, float xh, float xl) {
        float h, r, q;
        two_prod(ah, xh, h, r);
        two_sum(p, h, p, q);
        c = __fadd_rn(c, __fadd_rn(q, r));
        c = __fmaf_rn(ah, xl, c);
        c = __fmaf_rn(al, xh, c);
    }
    __device__ __forceinline__ double value() const { return f32_to_f64(p) + f32_to_f64(c); }
};

// v = hi + lo to ~48 bits (relative error <= 2e-15), on the integer pipes alone: hi is v rounded to
// FP32 (fastcvt.h) and lo the exact remainder -- the 29 mantissa bits below hi's, less 2^29 when
// hi rounded up, in units of v's last place -- normalised with a count of leading zeros and
// rounded to 24 bits.  lo is 0 where hi is 0 or infinite (|v| outside [2^-126, 2^128)) and where
// the remainder falls below 2^-126.
__device__ __forceinline__ void split(double v, float& hi, float& lo) {
    const unsigned hw = (unsigned)__double2hiint(v), lw = (unsigned)__double2loint(v);
    hi = f64_to_f32(v);
    const int e11 = (int)((hw & 0x7FFFFFFFu) >> 20);
    const int r = (int)(lw & 0x1FFFFFFFu) - (int)((lw >> 28) & 1u) * (1 << 29);
    const unsigned a = (unsigned)(r < 0 ? -r : r);   // < 2^29
    const int p = 31 - __clz(a);                      // its top bit
    const int sh = p - 23;
    const unsigned mant = sh > 0 ? (((a >> (sh - 1)) + 1u) >> 1) : (a << (-sh));   // in [2^23, 2^24]
    const int e8 = e11 + p - 948;                     // (e11 - 1075) + p + 127
    unsigned bits = ((hw & 0x80000000u) ^ (r < 0 ? 0x80000000u : 0u)) | (unsigned)((e8 << 23) + (int)mant - (1 << 23));
    bits = (a == 0u || e8 <= 0 || e11 <= 896 || e11 >= 1151) ? 0u : bits;
    lo = __uint_as_float(bits);
}

}  // namespace hdgdg
