// Double-float ("df64") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2, which
// carries a 48-bit significand.  GB300 issues FP32 instructions at 58x the rate of FP64
// ones (measured), so level-1 vectors of the mixed-precision solve are stored as (hi, lo)
// pairs -- 8 bytes per element, as FP64 -- and their Arnoldi arithmetic runs in FP32.
//
// The building blocks are the classical error-free transformations: Knuth's TwoSum (the
// rounding error of a sum is itself a float), Dekker's Fast2Sum for |a| >= |b|, and the
// FMA form of TwoProduct (fmaf(a, b, -a*b) is the exact error of a*b).  Products drop the
// lo*lo term (relative 2^-48).  nvcc does not reassociate float arithmetic, and the only
// contractions used are the explicit fmaf calls.
#pragma once

#include <cuda_runtime.h>

namespace mk {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {
    float s = a + b;
    float e = b - (s - a);
    return {s, e};
}

__device__ __forceinline__ df two_prod(float a, float b) {
    float p = a * b;
    float e = fmaf(a, b, -p);
    return {p, e};
}

// x + y (both double-float), error O(2^-46) relative
__device__ __forceinline__ df df_add(df x, df y) {
    df s = two_sum(x.hi, y.hi);
    s.lo += x.lo + y.lo;
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }

__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

// x * y with y a float
__device__ __forceinline__ df df_mul_f(df x, float y) {
    df p = two_prod(x.hi, y);
    p.lo = fmaf(x.lo, y, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

// x * y (both double-float)
__device__ __forceinline__ df df_mul(df x, df y) {
    df p = two_prod(x.hi, y.hi);
    p.lo = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo));
    return fast_two_sum(p.hi, p.lo);
}

// a + b for floats (exact)
__device__ __forceinline__ df df_from_sum(float a, float b) { return two_sum(a, b); }

__device__ __forceinline__ df df_from_float(float a) { return {a, 0.f}; }

// (l - 2 c + r) of three floats, exactly, as a double-float (two TwoSums; -2 c is exact)
__device__ __forceinline__ df lap3_exact(float l, float c, float r) {
    const df s1 = two_sum(l, r);
    const df s2 = two_sum(s1.hi, -2.f * c);
    return fast_two_sum(s2.hi, s2.lo + s1.lo);
}

// (l + r) + (d + u) - 4 c of five floats as a double-float: the pair sums exact, their sum
// and the -4 c term with roundings of order 2^-48 of the largest operand
__device__ __forceinline__ df lap5_df(float l, float r, float d, float u, float c) {
    const df s = df_add(two_sum(l, r), two_sum(d, u));
    const df t = two_sum(s.hi, -4.f * c);
    return fast_two_sum(t.hi, t.lo + s.lo);
}

// (l + r) + (d + u) - 4 c of five floats as an unnormalised pair (hi, lo): the leading sums
// by TwoSum, their four rounding errors added in FP32 (error of order 2^-47 of the largest
// operand; the pair is renormalised by whatever consumes it)
__device__ __forceinline__ df lap5_pair(float l, float r, float d, float u, float c) {
    const df a = two_sum(l, r), b = two_sum(d, u);
    const df s = two_sum(a.hi, b.hi);
    const df t = two_sum(s.hi, -4.f * c);
    return {t.hi, ((a.lo + b.lo) + s.lo) + t.lo};
}

// a x + b y of double-float operands (x, y possibly unnormalised), renormalised once by its
// consumer: the leading products exact (TwoProduct), their sum by TwoSum, the cross terms
// a.hi x.lo + a.lo x.hi (and for b, y) and the errors in FP32; the lo*lo terms are dropped
// (relative 2^-48)
__device__ __forceinline__ df df_dot2(df a, df x, df b, df y) {
    const df p = two_prod(a.hi, x.hi), q = two_prod(b.hi, y.hi);
    const df s = two_sum(p.hi, q.hi);
    const float lo = fmaf(a.hi, x.lo, fmaf(a.lo, x.hi, p.lo)) + fmaf(b.hi, y.lo, fmaf(b.lo, y.hi, q.lo));
    return {s.hi, s.lo + lo};
}
__device__ __forceinline__ df df_dot1(df a, df x) {
    const df p = two_prod(a.hi, x.hi);
    return {p.hi, fmaf(a.hi, x.lo, fmaf(a.lo, x.hi, p.lo))};
}

// (c - p) - D for floats c, p and a double-float D (possibly unnormalised): c - p exact by
// TwoSum, one TwoSum with D.hi, the low parts in FP32, one renormalisation
__device__ __forceinline__ df df_diff_sub(float c, float p, df D) {
    const df d = two_sum(c, -p);
    const df e = two_sum(d.hi, -D.hi);
    return fast_two_sum(e.hi, (d.lo - D.lo) + e.lo);
}

__host__ __device__ __forceinline__ float2 df_pack(df x) { return make_float2(x.hi, x.lo); }
__host__ __device__ __forceinline__ df df_unpack(float2 v) { return {v.x, v.y}; }

// conversions with FP64 (FP64 pipe; used once per restart, not in the inner loops)
__device__ __forceinline__ df df_from_double(double d) {
    float hi = (float)d;
    float lo = (float)(d - (double)hi);
    return {hi, lo};
}
__device__ __forceinline__ double df_to_double(df x) { return (double)x.hi + (double)x.lo; }

inline float2 df_pack_host(double d) {
    float hi = (float)d;
    float lo = (float)(d - (double)hi);
    return make_float2(hi, lo);
}

}  // namespace mk
