// Double-float ("df") arithmetic: a value is the unevaluated sum hi + lo of
// two floats, carrying about 48 significant bits with FP32 instructions only.
//
// GB300 issues FP64 at roughly 1/64 of its FP32 rate, so libpcal keeps FP64
// for the per-bin decode and rotation and uses df sums wherever many values
// are combined (reductions, prefix sums, the least-squares delay fit).
//
// The building blocks are the classical error-free transformations:
//   two_sum       Knuth's TwoSum: s + e == a + b exactly (6 flops);
//   quick_two_sum Dekker's Fast2Sum, valid when |a| >= |b| (3 flops);
//   two_prod      p + e == a * b exactly, with one fused multiply-add;
// and the df add / multiply / divide / square root built from them in the
// usual way (Dekker 1971; Shewchuk 1997; Hida, Li and Bailey 2001).
#pragma once

#include <math.h>

#ifndef PCAL_HD
#if defined(__CUDACC__)
#define PCAL_HD __host__ __device__ __forceinline__
#else
#define PCAL_HD inline
#endif
#endif

namespace pcal_df {

struct df {
    float hi, lo;
};

PCAL_HD df make(float hi, float lo = 0.0f) { return df{hi, lo}; }

PCAL_HD df two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return df{s, e};
}

PCAL_HD df quick_two_sum(float a, float b) {
    const float s = a + b;
    return df{s, b - (s - a)};
}

PCAL_HD df two_prod(float a, float b) {
    const float p = a * b;
    return df{p, fmaf(a, b, -p)};
}

PCAL_HD df neg(df x) { return df{-x.hi, -x.lo}; }

// Accurate df + df (both pairs of parts are summed error-free).
PCAL_HD df add(df x, df y) {
    df s = two_sum(x.hi, y.hi);
    const df t = two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}

PCAL_HD df add_f(df x, float y) {
    df s = two_sum(x.hi, y);
    s.lo += x.lo;
    return quick_two_sum(s.hi, s.lo);
}

PCAL_HD df sub(df x, df y) { return add(x, neg(y)); }

PCAL_HD df mul(df x, df y) {
    df p = two_prod(x.hi, y.hi);
    p.lo += x.hi * y.lo + x.lo * y.hi;
    return quick_two_sum(p.hi, p.lo);
}

PCAL_HD df mul_f(df x, float y) {
    df p = two_prod(x.hi, y);
    p.lo += x.lo * y;
    return quick_two_sum(p.hi, p.lo);
}

// Approximate float quotient; the df steps below correct its error.
PCAL_HD float fdiv_approx(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fdividef(a, b);
#else
    return a / b;
#endif
}

// x / y by two correction steps of an approximate float quotient.
PCAL_HD df div(df x, df y) {
    const float q1 = fdiv_approx(x.hi, y.hi);
    df r = sub(x, mul_f(y, q1));
    const float q2 = fdiv_approx(r.hi, y.hi);
    r = sub(r, mul_f(y, q2));
    const float q3 = fdiv_approx(r.hi, y.hi);
    return add_f(quick_two_sum(q1, q2), q3);
}

// sqrt(x) by one Newton correction of the float root; 0 for x <= 0.
PCAL_HD df sqrt_df(df x) {
    if (!(x.hi > 0.0f)) return df{0.0f, 0.0f};
    const float s = sqrtf(x.hi);
    const df r = sub(x, two_prod(s, s));
    return quick_two_sum(s, fdiv_approx(r.hi, 2.0f * s));
}

}  // namespace pcal_df
