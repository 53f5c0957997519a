// df.cuh -- double-float ("float-float") arithmetic on the FP32 pipe.
//
// A value is hi + lo with two floats, |lo| <= ulp(hi) / 2, about 48
// significant bits.  GB300 runs FP32 FMA ~73x faster than FP64 FMA, so the
// bulk arithmetic of the fast path (correlation tables, Gaussian weights,
// candidate screening) runs here, with FP64 kept for the few operations that
// combine partial results.
//
// Error-free transformations: Knuth's TwoSum, Dekker's Fast2Sum and the
// FMA-based TwoProd (see Joldes, Muller and Popescu, "Tight and rigorous
// error bounds for basic building blocks of double-word arithmetic", ACM
// TOMS 2017).  Rounded products use __fmul_rn so that no multiply-add is
// formed across an error-free transformation.  With u = 2^-24:
//   df_add     |err| <= 2 u^2 (|a| + |b|)
//   df_add_acc |err| <= 3 u^2 |a + b|
//   df_mul     |err| <= 5 u^2 |a b|
#pragma once

#include <cuda_runtime.h>

namespace ucp {

struct dfloat {
    float hi, lo;
};

__host__ __device__ inline dfloat df_from_double(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

__host__ __device__ inline double df_to_double(dfloat a) {
    return (double)a.hi + (double)a.lo;
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dfloat df_norm(float h, float l) {
    dfloat r;
    fast_two_sum(h, l, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return df_norm(s, e);
}

// Accurate addition (Joldes, Muller, Popescu, Algorithm 6): relative error
// <= 3 u^2 of the result, so small sums of large operands stay accurate.
__device__ __forceinline__ dfloat df_add_acc(dfloat a, dfloat b) {
    float sh, sl, th, tl;
    two_sum(a.hi, b.hi, sh, sl);
    two_sum(a.lo, b.lo, th, tl);
    const float c = __fadd_rn(sl, th);
    float vh, vl;
    fast_two_sum(sh, c, vh, vl);
    const float w = __fadd_rn(tl, vl);
    return df_norm(vh, w);
}

__device__ __forceinline__ dfloat df_add_f(dfloat a, float b) {
    float s, e;
    two_sum(a.hi, b, s, e);
    e = __fadd_rn(e, a.lo);
    return df_norm(s, e);
}

__device__ __forceinline__ dfloat df_neg(dfloat a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ dfloat df_sub(dfloat a, dfloat b) {
    return df_add(a, df_neg(b));
}

__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_norm(p, e);
}

__device__ __forceinline__ dfloat df_mul_f(dfloat a, float b) {
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return df_norm(p, e);
}

// Product a*b as an unnormalised pair (p, e) with p + e = a*b + O(5u^2|ab|).
__device__ __forceinline__ void df_mul_raw(dfloat a, dfloat b, float& p, float& e) {
    p = __fmul_rn(a.hi, b.hi);
    e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
}

// acc += (p + e), result normalised.
__device__ __forceinline__ dfloat df_acc(dfloat acc, float p, float e) {
    float s, t;
    two_sum(acc.hi, p, s, t);
    t = __fadd_rn(t, __fadd_rn(acc.lo, e));
    return df_norm(s, t);
}

// Exact double-float of an integer below 2^44 in magnitude, from two 32-bit
// conversions (64-bit integer conversions run on the FP64 pipe).
__device__ __forceinline__ dfloat df_from_i64(long long m) {
    const int hi = (int)(m >> 22);              // |hi| < 2^22
    const int lo = (int)(m & ((1 << 22) - 1));  // [0, 2^22)
    return df_norm(__int2float_rn(hi) * 4194304.0f, __int2float_rn(lo));
}

__device__ __forceinline__ bool df_lt(dfloat a, dfloat b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}

// exp(x) for a double-float x in [-87, 87]; relative error about 1e-14.
// Cody-Waite reduction x = n ln2 + r with ln2 split as C1 + C2 + C3 (C1 has
// 15 significant bits, so n C1 and x_hi - n C1 are exact), r = k/64 + s with
// |s| <= 1/128, exp(k/64) from the table `t64` (index k + 23, 47 entries), and
// exp(s) = 1 + s + s^2 (1/2 + s/6 + s^2/24 + s^3/120 + s^4/720).
__device__ __forceinline__ dfloat df_exp(dfloat x, const dfloat* __restrict__ t64) {
    const float C1 = 0.693145751953125f;
    const float C2 = 1.428606765330187e-06f;
    const float C3 = 5.497923148104107e-14f;
    const float n = rintf(__fmul_rn(x.hi, 1.44269502f));
    const float r0 = __fsub_rn(x.hi, __fmul_rn(n, C1));  // exact
    dfloat r;
    two_sum(r0, x.lo, r.hi, r.lo);
    r = df_norm(r.hi, r.lo);
    const float p = __fmul_rn(n, C2);
    const float pe = __fmaf_rn(n, C2, -p);
    r = df_add(r, dfloat{-p, -pe});
    r = df_add_f(r, -__fmul_rn(n, C3));
    const float k = rintf(__fmul_rn(r.hi, 64.0f));
    const dfloat s = df_norm(__fsub_rn(r.hi, __fmul_rn(k, 0.015625f)), r.lo);
    // g = 1/6 + s (1/24 + s (1/120 + s / 720)) with the bracket in float
    float q = __fmaf_rn(s.hi, 1.0f / 720.0f, 1.0f / 120.0f);
    q = __fmaf_rn(q, s.hi, 1.0f / 24.0f);
    const dfloat g = df_add_f(dfloat{0.1666666716337204f, -4.967053879312289e-09f},
                              __fmul_rn(s.hi, q));
    const dfloat h = df_add_f(df_mul(s, g), 0.5f);
    const dfloat es = df_add(df_add_f(s, 1.0f), df_mul(df_mul(s, s), h));
    dfloat v = df_mul(es, t64[(int)k + 23]);
    const float sc = __int_as_float((int)(127 + (int)n) << 23);
    return {__fmul_rn(v.hi, sc), __fmul_rn(v.lo, sc)};
}

}  // namespace ucp
