// Double-precision products and sums evaluated with FP32 arithmetic ("double-float").
//
// On GB300 the FP64 pipe issues ~0.5 G warp-lane operations per second per GPU (a few
// per SM per clock) against ~37 T for FP32 FMA, so an FP64 SpMV that spends even one FP64
// instruction per nonzero is bound by the FP64 pipe rather than by HBM.  The products
// a * x of the FP64 path are therefore formed from float pairs:
//   * a double a in the window [2^-50, 2^45] (or 0) splits exactly-enough into
//     hi = a with its mantissa truncated to 24 bits and lo = the remaining 29 mantissa
//     bits rounded to 24 (integer operations only; |a - hi - lo| <= 2^-48 |a|);
//   * a * x = ah*xh + [fma error of ah*xh] + ah*xl + al*xh  (the error-free product of
//     Dekker/Ogita-Rump-Oishi via FMA; al*xl ~ 2^-48 is dropped);
//   * the running sum is a float pair (s, c): s collects the rounded terms and c the
//     exact TwoSum errors (Knuth) plus the product corrections -- a compensated sum in the
//     style of Neumaier, with relative error ~2^-47 of the sum of |terms|.
// The window keeps every intermediate normal in FP32 (products in [2^-100, 2^90], sums of
// up to 2^31 terms below 2^121).  Values outside it make the caller use native FP64.
// All arithmetic uses the _rn intrinsics so that no step is contracted into an FMA.
#pragma once
#include <stdint.h>

namespace spmv {

constexpr uint32_t DF_EXP_MIN = 1023 - 50;   // biased double exponent window
constexpr uint32_t DF_EXP_MAX = 1023 + 45;

// Split a double into (hi, lo); returns false if a is nonzero and outside the window.
__device__ __forceinline__ bool df_split(double a, float *hi, float *lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(a);
    const uint32_t h32 = (uint32_t)(b >> 32), l32 = (uint32_t)b;
    const uint32_t E = (h32 >> 20) & 0x7FFu;
    if (((h32 & 0x7FFFFFFFu) | l32) == 0u) {
        *hi = 0.f;
        *lo = 0.f;
        return true;
    }
    const bool ok = E >= DF_EXP_MIN && E <= DF_EXP_MAX;
    const uint32_t Ec = ok ? E : 1023u;   // keep the bit patterns finite when out of range
    const uint32_t sign = h32 & 0x80000000u;
    *hi = __uint_as_float(sign | ((Ec - 896u) << 23) | ((h32 & 0xFFFFFu) << 3) | (l32 >> 29));
    const float scale = __uint_as_float((Ec - 948u) << 23);   // 2^(E - 1075)
    *lo = __uint_as_float(__float_as_uint(__fmul_rn(__uint2float_rn(l32 & 0x1FFFFFFFu), scale)) | sign);
    return ok;
}

// (s, c) += a * x with a = (ah, al), x = (xh, xl).
__device__ __forceinline__ void df_fma(float ah, float al, float xh, float xl, float &s, float &c) {
    const float p = __fmul_rn(ah, xh);
    float pe = __fmaf_rn(ah, xh, -p);
    pe = __fmaf_rn(ah, xl, pe);
    pe = __fmaf_rn(al, xh, pe);
    const float t = __fadd_rn(s, p);
    const float bp = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, pe));
}

// (s, c) += (t, d)
__device__ __forceinline__ void df_add(float &s, float &c, float t, float d) {
    const float u = __fadd_rn(s, t);
    const float bp = __fsub_rn(u, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(u, bp)), __fsub_rn(t, bp));
    s = u;
    c = __fadd_rn(__fadd_rn(c, d), e);
}

// Exact float -> double widening with integer operations (zero and subnormals take the
// conversion instruction).
__device__ __forceinline__ double df_widen(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu;
    if (e == 0u || e == 0xFFu) return (double)f;
    const unsigned long long d = ((unsigned long long)(u & 0x80000000u) << 32) |
                                 ((unsigned long long)(e + 896u) << 52) |
                                 ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)d);
}

// The same for normal numbers and zeros only, in 32-bit operations: the double's high word holds
// the sign, the exponent rebiased by 1023 - 127 = 896 and the top 20 mantissa bits, the low word
// the last 3 mantissa bits.
__device__ __forceinline__ double df_widen_normal(float f) {
    const uint32_t u = __float_as_uint(f), mag = u & 0x7FFFFFFFu;
    const uint32_t hi = mag == 0u ? 0u : (mag >> 3) + (896u << 20);
    return __hiloint2double((int)(hi | (u & 0x80000000u)), (int)(u << 29));
}

// A subnormal, infinite or NaN float (the classes df_widen_normal does not cover).
__device__ __forceinline__ bool df_special(float f) {
    const uint32_t mag = __float_as_uint(f) & 0x7FFFFFFFu;
    return mag != 0u && mag - 0x00800000u >= 0x7F000000u;
}

// (s, c) as one double: one FP64 addition of the exactly widened parts.  The short widening
// serves every lane unless a lane of the warp holds a special part (the result is the same
// either way: both widenings are exact).
__device__ __forceinline__ double df_to_double(float s, float c) {
    if (__any_sync(__activemask(), df_special(s) || df_special(c))) return df_widen(s) + df_widen(c);
    return df_widen_normal(s) + df_widen_normal(c);
}

}  // namespace spmv
