// smap_df.cuh -- double-float ("df") arithmetic on the FP32 pipe.
//
// A df value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2: about 48 significant bits, built from FP32 adds and
// FMAs by error-free transformations (Dekker 1971, "A floating-point
// technique for extending the available precision"; Knuth's TwoSum, TAOCP
// vol. 2, 4.2.2; the exact rounding error of a product from one FMA). GB300
// issues FP64 at 1/64 of the FP32 rate, so the per-particle terms of the
// recursion's FP64 scores (log-likelihood and transition density) are
// evaluated here and only the accumulation into phi stays in FP64.
//
// Every operation uses the explicitly rounded intrinsics (__fadd_rn, ...),
// which the compiler neither contracts into FMAs nor reorders.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace smap {
namespace df {

struct F {
    float hi, lo;
};

__device__ __forceinline__ F make(float hi, float lo) { return F{hi, lo}; }

// s + e = a + b exactly (any magnitudes).
__device__ __forceinline__ F two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return F{s, e};
}
// The same when |a| >= |b| (or a = 0).
__device__ __forceinline__ F fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return F{s, __fsub_rn(b, __fsub_rn(s, a))};
}
// p + e = a b exactly.
__device__ __forceinline__ F two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return F{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ F neg(F a) { return F{-a.hi, -a.lo}; }
// Exact scaling by a power of two (no overflow or underflow in use here).
__device__ __forceinline__ F scale2(F a, float p2) { return F{__fmul_rn(a.hi, p2), __fmul_rn(a.lo, p2)}; }

__device__ __forceinline__ F add(F a, F b) {
    F s = two_sum(a.hi, b.hi);
    const F t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ F sub(F a, F b) { return add(a, neg(b)); }
__device__ __forceinline__ F add_f(F a, float b) {
    F s = two_sum(a.hi, b);
    s.lo = __fadd_rn(s.lo, a.lo);
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ F mul(F a, F b) {
    F p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
    p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
    return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ F mul_f(F a, float b) {
    F p = two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ F sqr(F a) {
    F p = two_prod(a.hi, a.hi);
    p.lo = __fmaf_rn(__fadd_rn(a.hi, a.hi), a.lo, p.lo);
    return fast_two_sum(p.hi, p.lo);
}
// a / b: the FP32 quotient corrected once by the df remainder a - q b.
__device__ __forceinline__ F div(F a, F b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const F r = sub(a, mul_f(b, q1));
    const float q2 = __fdiv_rn(r.hi, b.hi);
    return fast_two_sum(q1, q2);
}
__device__ __forceinline__ double to_double(F a) { return (double)a.hi + (double)a.lo; }

// sqrt(a), a > 0: the FP32 root y corrected once by (a - y^2) / (2 y), with
// a - y^2 formed exactly (Karp and Markstein 1997, "High-precision division
// and square root").
__device__ __forceinline__ F sqrt(F a) {
    const float y = sqrtf(a.hi);
    const F y2 = two_prod(y, y);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, y2.hi), y2.lo), a.lo);
    return fast_two_sum(y, __fdiv_rn(r, __fadd_rn(y, y)));
}

// p = c + x q in df (one Horner step).
__device__ __forceinline__ F horner(F q, F x, F c) { return add(mul(q, x), c); }

// exp(t) for -60 < t < 60 (further out the low part of the result leaves
// FP32's normal range): t = k ln2 + r with ln 2 split into three parts
// (the first exactly multiplied by the integer k, the second by an exact
// product), |r| <= ln2/2; x = r/2 goes into the Taylor series (orders 7-11 in
// FP32, where they are below 2^-27 of the sum; orders 0-6 in df), and the
// result is squared once and scaled by 2^k.
__device__ __forceinline__ F exp(F t) {
    const float k = rintf(__fmul_rn(t.hi, 1.4426950408889634f));
    // ln 2 = L1 + L2 + L3; L1 has 16 significant bits (k L1 is exact for |k| < 256)
    const float L1 = 0.693145751953125f, L2 = 1.428606765330187e-06f, L3 = 5.497923148104107e-14f;
    F r = add_f(t, -__fmul_rn(k, L1));
    r = sub(r, two_prod(k, L2));
    r = add_f(r, -__fmul_rn(k, L3));
    const F x = scale2(r, 0.5f);
    const float xf = x.hi;
    // 1/7! + x/8! + x^2/9! + x^3/10! + x^4/11!
    float v = __fmaf_rn(xf, 2.5052108385441720e-08f, 2.7557319223985893e-07f);
    v = __fmaf_rn(xf, v, 2.7557319223985891e-06f);
    v = __fmaf_rn(xf, v, 2.4801587301587302e-05f);
    v = __fmaf_rn(xf, v, 1.9841269841269841e-04f);
    F q = add(mul_f(x, v), make(0.0013888889225199819f, -3.3631094437103215e-11f));   // 1/6!
    q = horner(q, x, make(0.008333333767950535f, -4.34617203337595e-10f));           // 1/5!
    q = horner(q, x, make(0.0416666679084301f, -1.2417634698280722e-09f));            // 1/4!
    q = horner(q, x, make(0.1666666716337204f, -4.967053879312289e-09f));             // 1/3!
    q = horner(q, x, make(0.5f, 0.0f));
    q = horner(q, x, make(1.0f, 0.0f));
    q = horner(q, x, make(1.0f, 0.0f));
    q = sqr(q);
    return scale2(q, __int_as_float((127 + (int)k) << 23));
}

// log(a), a > 0 normal: a = 2^e m with m in [sqrt(1/2), sqrt(2)), z = (m - 1) /
// (m + 1), log m = 2 atanh z = 2 z (1 + w/3 + w^2/5 + ...), w = z^2 <= 0.0295
// (orders w^5 .. w^9 in FP32, where they are below 2^-28 of the sum; the
// lower ones in df), plus e ln 2.
__device__ __forceinline__ F log(F a) {
    int e = (int)((__float_as_uint(a.hi) >> 23) & 0xff) - 127;
    F m = scale2(a, __int_as_float((uint32_t)(127 - e) << 23));   // a 2^-e in [1, 2)
    if (m.hi > 1.4142135623730951f) {
        m = scale2(m, 0.5f);
        e += 1;
    }
    const F z = div(add_f(m, -1.0f), add_f(m, 1.0f));
    const F w = sqr(z);
    const float wf = w.hi;
    // 1/11 + w/13 + w^2/15 + w^3/17 + w^4/19
    float v = __fmaf_rn(wf, 5.2631578947368421e-02f, 5.8823529411764705e-02f);
    v = __fmaf_rn(wf, v, 6.6666666666666667e-02f);
    v = __fmaf_rn(wf, v, 7.6923076923076923e-02f);
    v = __fmaf_rn(wf, v, 9.0909090909090909e-02f);
    F q = add(mul_f(w, v), make(0.1111111119389534f, -8.278422947149977e-10f));       // 1/9
    q = horner(q, w, make(0.1428571492433548f, -6.38621200366174e-09f));              // 1/7
    q = horner(q, w, make(0.20000000298023224f, -2.9802322831784522e-09f));           // 1/5
    q = horner(q, w, make(0.3333333432674408f, -9.934107758624577e-09f));             // 1/3
    q = horner(q, w, make(1.0f, 0.0f));
    q = scale2(mul(q, z), 2.0f);
    return add(q, mul_f(make(0.6931471824645996f, -1.9046542121259336e-09f), (float)e));   // + e ln 2
}

}  // namespace df
}  // namespace smap
