// Double-float arithmetic: a value held as an unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi) / 2 (48 significant bits, FP32's exponent range).
// The building blocks are the error-free transformations of Dekker (1971) and Knuth
// (TAOCP vol. 2, Sec. 4.2.2): TwoSum (s + t = a + b exactly, any order of magnitude),
// FastTwoSum (the same for |a| >= |b|, three operations) and the FMA form of
// TwoProduct (p + e = a b exactly).  The products drop the lo x lo term and round the
// two cross terms into e, so a product or multiply-add has a relative error of a few
// units of 2^-48.  Every operation goes through the round-to-nearest intrinsics so
// that the compiler neither contracts an addition with a product into an FMA nor
// reorders them (either would break the exactness that the error terms rely on).
//
// The bulge chasing of the mixed path runs in this arithmetic on the FP32 pipe, whose
// throughput on GB300 is about 70 times that of its FP64 pipe.
#pragma once

#include <cuda_runtime.h>

struct __align__(8) df32 {
    float hi, lo;
};

__device__ __forceinline__ df32 df_make(float hi, float lo) {
    df32 r;
    r.hi = hi;
    r.lo = lo;
    return r;
}

// FP64 -> double-float (hi the FP64 value rounded to FP32, lo the rest rounded)
__device__ __forceinline__ df32 df_from_double(double x) {
    const float h = __double2float_rn(x);
    return df_make(h, __double2float_rn(x - (double)h));
}

// double-float -> FP64 (exact: the 48 bits of hi + lo fit in FP64's 53)
__device__ __forceinline__ double df_to_double(df32 a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df32 df_neg(df32 a) { return df_make(-a.hi, -a.lo); }

// Knuth's TwoSum: s = fl(a + b), t = (a + b) - s exactly
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& t) {
    s = __fadd_rn(a, b);
    const float bb = __fadd_rn(s, -a);
    t = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
}

// Dekker's FastTwoSum, renormalising (s, t) with |s| >= |t|
__device__ __forceinline__ df32 df_fast_two_sum(float s, float t) {
    const float h = __fadd_rn(s, t);
    return df_make(h, __fadd_rn(t, -__fadd_rn(h, -s)));
}

// a b as an unevaluated p + e (TwoProduct on hi x hi, cross terms folded into e)
__device__ __forceinline__ void df_prod_terms(df32 a, df32 b, float& p, float& e) {
    p = __fmul_rn(a.hi, b.hi);
    e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
}

// a + b
__device__ __forceinline__ df32 df_add(df32 a, df32 b) {
    float s, t;
    df_two_sum(a.hi, b.hi, s, t);
    t = __fadd_rn(t, __fadd_rn(a.lo, b.lo));
    return df_fast_two_sum(s, t);
}

// a b
__device__ __forceinline__ df32 df_mul(df32 a, df32 b) {
    float p, e;
    df_prod_terms(a, b, p, e);
    return df_fast_two_sum(p, e);
}

// c + a b
__device__ __forceinline__ df32 df_fma(df32 a, df32 b, df32 c) {
    float p, e, s, t;
    df_prod_terms(a, b, p, e);
    df_two_sum(c.hi, p, s, t);
    t = __fadd_rn(t, __fadd_rn(c.lo, e));
    return df_fast_two_sum(s, t);
}

// c - a b - d e' (two products subtracted with one renormalisation)
__device__ __forceinline__ df32 df_sub2(df32 c, df32 a, df32 b, df32 d, df32 f) {
    float p1, e1, p2, e2, s, t, s2, t2;
    df_prod_terms(a, b, p1, e1);
    df_prod_terms(d, f, p2, e2);
    df_two_sum(c.hi, -p1, s, t);
    t = __fadd_rn(t, __fadd_rn(c.lo, -e1));
    df_two_sum(s, -p2, s2, t2);
    t2 = __fadd_rn(t2, __fadd_rn(t, -e2));
    return df_fast_two_sum(s2, t2);
}

// Running sum of products in the style of Ogita, Rump & Oishi's Dot2 (SIAM J. Sci.
// Comput. 26, 2005): the FP32 sum s takes each product's leading part through TwoSum,
// and c collects the sum's and the products' error terms; s + c is the value.  Only s
// carries a dependency from one term to the next (one addition), so long dot products
// are not bound by the latency of a renormalisation per term.
struct df_acc {
    float s, c;
};
__device__ __forceinline__ df_acc df_acc_zero() {
    df_acc a;
    a.s = 0.0f;
    a.c = 0.0f;
    return a;
}
__device__ __forceinline__ void df_acc_add(df_acc& acc, df32 a, df32 b) {
    float p, e, s, t;
    df_prod_terms(a, b, p, e);
    df_two_sum(acc.s, p, s, t);
    acc.s = s;
    acc.c = __fadd_rn(acc.c, __fadd_rn(t, e));
}
__device__ __forceinline__ df32 df_acc_value(df_acc a) { return df_fast_two_sum(a.s, a.c); }
__device__ __forceinline__ df32 df_acc_merge(df_acc a, df_acc b) {
    float s, t;
    df_two_sum(a.s, b.s, s, t);
    return df_fast_two_sum(s, __fadd_rn(t, __fadd_rn(a.c, b.c)));
}

// square root of a >= 0: the FP32 root corrected by one Newton step on the remainder
// a - x^2 computed in double-float (Karp & Markstein, ACM TOMS 23, 1997)
__device__ __forceinline__ df32 df_sqrt(df32 a) {
    if (!(a.hi > 0.0f)) return df_make(0.0f, 0.0f);
    const float x = sqrtf(a.hi);
    const float p = __fmul_rn(x, x), e = __fmaf_rn(x, x, -p);  // x^2 = p + e exactly
    // a.hi - p is exact (the two are within a factor of two of each other)
    const float r = __fadd_rn(__fadd_rn(__fadd_rn(a.hi, -p), -e), a.lo);
    return df_fast_two_sum(x, __fdiv_rn(r, __fmul_rn(2.0f, x)));
}

// a / b: the FP32 quotient q1 corrected by the quotient of the remainder a - q1 b
// (Dekker's double-length division, Numer. Math. 18, 1971)
__device__ __forceinline__ df32 df_div(df32 a, df32 b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    float p, e, s, t;
    p = __fmul_rn(q1, b.hi);
    e = __fmaf_rn(q1, b.hi, -p);
    e = __fmaf_rn(q1, b.lo, e);
    df_two_sum(a.hi, -p, s, t);
    t = __fadd_rn(t, __fadd_rn(a.lo, -e));
    return df_fast_two_sum(q1, __fdiv_rn(__fadd_rn(s, t), b.hi));
}

__device__ __forceinline__ df32 df_shfl(df32 a, int src) {
    return df_make(__shfl_sync(0xffffffffu, a.hi, src), __shfl_sync(0xffffffffu, a.lo, src));
}

// sum over the warp (butterfly: every lane adds the same pairs, so all lanes agree)
__device__ __forceinline__ df32 df_warp_sum(df32 a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        a = df_add(a, df_make(__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)));
    return a;
}
