// Exact FP32 splitting of FP64 values and error-free FP32 transformations, for the arithmetic
// of the mixed-precision form that must keep FP64-grade accuracy off the FP64 pipe (which on
// this GPU retires 2 lanes per SM per clock against 128 for FP32).
#pragma once

#include <cuda_runtime.h>

namespace tc {
namespace xs {

// (hi, lo) with hi = d truncated to 24 significant bits and lo = the next 23 bits of d, both
// read off the bit pattern: |d - hi - lo| < 2^-46 |d|.  |d| < 2^-126 gives (0, 0), which is
// below any value the state carries at a resolvable level; |d| >= 2^128 gives +-inf and NaN
// stays NaN, so a non-finite state still shows in the output.
__device__ __forceinline__ float2 split_hl(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned int h = (unsigned int)(b >> 32);
    const unsigned int l = (unsigned int)b;
    const unsigned int s = h & 0x80000000u;
    const int e = (int)((h >> 20) & 0x7ffu);
    float2 r;
    if (e <= 896) {
        r.x = 0.f;
        r.y = 0.f;
        return r;
    }
    if (e >= 1151) {
        const bool nan = e == 2047 && (((h & 0xfffffu) | l) != 0u);
        r.x = __uint_as_float(s | 0x7f800000u | (nan ? 0x400000u : 0u));
        r.y = 0.f;
        return r;
    }
    const unsigned int top = ((h & 0xfffffu) << 3) | (l >> 29);
    r.x = __uint_as_float(s | ((unsigned int)(e - 896) << 23) | top);
    // low 29 mantissa bits have weight 2^(e - 1075); their top 23 (weight 2^(e - 1069)) as an
    // exact float: 2^23 + n has the bit pattern 0x4b000000 | n for n < 2^23
    const unsigned int rem = (l & 0x1fffffffu) >> 6;
    const float fr = __fsub_rn(__uint_as_float(0x4b000000u | rem), 8388608.0f);
    const int es = e - 942;   // biased FP32 exponent of 2^(e - 1069)
    const float sc = es > 0 ? __uint_as_float((unsigned int)es << 23) : 0.f;
    r.y = __uint_as_float(__float_as_uint(__fmul_rn(fr, sc)) | s);
    return r;
}

// FP32 -> FP64 by the bit pattern (exact; FP32 subnormals, never produced here, give 0)
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned int u = __float_as_uint(f);
    const unsigned int e = (u >> 23) & 0xffu;
    const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
    if (e == 0u) return __longlong_as_double((long long)s);
    const unsigned long long ed = e == 255u ? 2047ull : (unsigned long long)(e + 896u);
    const unsigned long long m = (unsigned long long)(u & 0x7fffffu) << 29;
    return __longlong_as_double((long long)(s | (ed << 52) | m));
}

// error-free transformations (Dekker's product via FMA, Knuth's sum); the _rn intrinsics keep
// the compiler from contracting them into FMAs
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + c += (ah + al)(bh + bl): the exact product of the high parts folded in by an error-free
// sum, the lower-order parts accumulated in c (compensated dot product, Ogita-Rump-Oishi)
__device__ __forceinline__ void dot_acc(float& s, float& c, float ah, float al, float bh, float bl) {
    float p, e, q;
    two_prod(ah, bh, p, e);
    e = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
    two_sum(s, p, s, q);
    c = __fadd_rn(c, __fadd_rn(q, e));
}

}  // namespace xs
}  // namespace tc
