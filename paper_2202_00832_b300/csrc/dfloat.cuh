// Double-float arithmetic: a value is hi + lo, two FP32 numbers, kept
// unevaluated.  B300 issues FP32 about 64x faster than FP64; an error-free
// product (FMA) and sum (Knuth TwoSum) carry about 48 significant bits.
#pragma once
#include <cuda_runtime.h>

namespace loaf {

// A complex double-float is a float4 {re.hi, re.lo, im.hi, im.lo}.
struct dfl {
    float hi, lo;
};
__device__ inline dfl df_from(double x) {
    dfl r;
    r.hi = (float)x;
    r.lo = (float)(x - (double)r.hi);
    return r;
}
__device__ inline double df_to(dfl a) { return (double)a.hi + (double)a.lo; }
// hi + lo = x (to about 2^-48 relative) from the bit pattern of x with FP32 and
// integer operations only: hi keeps the top 24 significand bits (truncated),
// lo the remaining 29, rounded to a float.  |x| within the float range.
__device__ inline dfl df_split_bits(double x) {
    const long long b = __double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff);
    // fast range: 2^(ex - 1075) (the unit of lo) and hi both normal floats
    if (ex < 1075 - 126 || ex > 1023 + 127) return df_from(x);
    const long long m = (b & 0xfffffffffffffLL) | 0x10000000000000LL;  // 53 bits
    const long long mh = m >> 29, ml = m & ((1LL << 29) - 1);
    const float sgn = b < 0 ? -1.f : 1.f;
    // x = (mh 2^29 + ml) 2^(ex - 1075)
    dfl r;
    r.hi = sgn * __int_as_float((int)((ex - 1023 + 127) << 23) | (int)(mh & 0x7fffff));
    r.lo = sgn * __fmul_rn(__int2float_rn((int)ml), __int_as_float((ex - 1075 + 127) << 23));
    return r;
}
__device__ inline dfl df_neg(dfl a) { return dfl{-a.hi, -a.lo}; }
// c + a b.  The _rn intrinsics are never contracted into FMAs, which would
// break the error-free sums.
__device__ inline dfl df_fma(dfl a, dfl b, dfl c) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);  // exact error of the product
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float s = __fadd_rn(c.hi, p);  // TwoSum(c.hi, p)
    const float v = __fsub_rn(s, c.hi);
    float t = __fadd_rn(__fsub_rn(c.hi, __fsub_rn(s, v)), __fsub_rn(p, v));
    t = __fadd_rn(t, c.lo);
    t = __fadd_rn(t, e);
    dfl r;
    r.hi = __fadd_rn(s, t);  // renormalise
    r.lo = __fsub_rn(t, __fsub_rn(r.hi, s));
    return r;
}
__device__ inline dfl df_mul(dfl a, dfl b) { return df_fma(a, b, dfl{0.f, 0.f}); }

// Two double-floats as the lanes of float2 pairs (hi, lo), e.g. the real and
// imaginary parts of a complex value: df2_fma is df_fma on both lanes, one
// sm_100 FP32x2 instruction per step (the same operations in the same order).
struct dfl2 {
    float2 hi, lo;
};
__device__ inline float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ inline dfl2 df2_fma(dfl2 a, dfl2 b, dfl2 c) {
    const float2 p = __fmul2_rn(a.hi, b.hi);
    float2 e = __ffma2_rn(a.hi, b.hi, neg2(p));  // exact error of the product
    e = __ffma2_rn(a.hi, b.lo, e);
    e = __ffma2_rn(a.lo, b.hi, e);
    const float2 s = __fadd2_rn(c.hi, p);  // TwoSum(c.hi, p)
    const float2 v = __fadd2_rn(s, neg2(c.hi));
    float2 t = __fadd2_rn(__fadd2_rn(c.hi, neg2(__fadd2_rn(s, neg2(v)))), __fadd2_rn(p, neg2(v)));
    t = __fadd2_rn(t, c.lo);
    t = __fadd2_rn(t, e);
    dfl2 r;
    r.hi = __fadd2_rn(s, t);  // renormalise
    r.lo = __fadd2_rn(t, neg2(__fadd2_rn(r.hi, neg2(s))));
    return r;
}

}  // namespace loaf
