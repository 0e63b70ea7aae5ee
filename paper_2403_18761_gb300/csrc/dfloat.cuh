// Double-float arithmetic: a value is hi + lo with two FP32 numbers
// (about 44 significant bits).  Used for piece volumes and moments in the
// FP32-filtered mode, where native FP64 (1/64 of the FP32 rate on this GPU)
// would dominate the clip kernel.  Built on the classical error-free
// transformations (Knuth's two-sum, Dekker's fast two-sum, and the FMA form of
// two-product).  The __f*_rn intrinsics keep the compiler from contracting or
// reassociating the operations.
#pragma once

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(float a) { return {a, 0.0f}; }

__device__ __forceinline__ df fast_two_sum(float a, float b) {   // needs |a| >= |b|
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df df_add(df x, df y) {
    df s = two_sum(x.hi, y.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

__device__ __forceinline__ df df_mul(df x, df y) {
    float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}

// a / b with one FP32 division and one correction step.
__device__ __forceinline__ df df_div(df a, df b) {
    float q1 = __fdiv_rn(a.hi, b.hi);
    df r = df_sub(a, df_mul(df_make(q1), b));
    float q2 = __fdiv_rn(r.hi, b.hi);
    return fast_two_sum(q1, q2);
}

// a / b from approximate FP32 quotients (about 2^-22 each) and one exact
// residual correction: relative error about 2^-44, the double-float level.
// Needs |b.hi| within the normal FP32 range.
__device__ __forceinline__ df df_div_fast(df a, df b) {
    const float q1 = __fdividef(a.hi, b.hi);
    const df r = df_sub(a, df_mul(df_make(q1), b));
    const float q2 = __fdividef(r.hi, b.hi);
    return fast_two_sum(q1, q2);
}

__device__ __forceinline__ double df_to_double(df x) { return (double)x.hi + (double)x.lo; }

// sqrt(x) for x >= 0 (0 otherwise): the FP32 root s and one Newton step on
// the exact residual x - s^2 (two-product by FMA), relative error about 2^-44.
__device__ __forceinline__ df df_sqrt(df x) {
    if (!(x.hi > 0.0f)) return {0.0f, 0.0f};
    const float s = __fsqrt_rn(x.hi);
    const float p = __fmul_rn(s, s);
    const float pe = __fmaf_rn(s, s, -p);   // s * s = p + pe exactly
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p), pe), x.lo);
    return fast_two_sum(s, __fdiv_rn(r, __fmul_rn(2.0f, s)));
}

// Exact conversion of |v| < 2^48 (two exactly representable parts).
__device__ __forceinline__ df df_from_i64(long long v) {
    long long h = v >> 24;                 // arithmetic shift: v = h * 2^24 + l, 0 <= l < 2^24
    long long l = v - (h << 24);
    return two_sum(__int2float_rn((int)h) * 16777216.0f, __int2float_rn((int)l));
}

__device__ __forceinline__ df df_scale(df x, float p2) { return {x.hi * p2, x.lo * p2}; }

// |v| < 2^127 to double-float: the top 48 bits exactly, the rest truncated
// (relative error below 2^-47).
__device__ __forceinline__ df df_from_i128(__int128 v) {
    const bool neg = v < 0;
    unsigned __int128 a = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
    const unsigned long long hi = (unsigned long long)(a >> 64), lo = (unsigned long long)a;
    const int len = hi ? 128 - __clzll((long long)hi) : 64 - (lo ? __clzll((long long)lo) : 64);
    const int sh = len > 48 ? len - 48 : 0;
    const long long top = (long long)(a >> sh);   // < 2^48
    df r = df_from_i64(neg ? -top : top);
    if (sh) r = df_scale(r, __int_as_float((127 + sh) << 23));
    return r;
}
