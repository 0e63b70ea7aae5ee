// Exact signed 256-bit integers for the last-resort clip predicates.
//
// A clip predicate is sign(F_u . C) where F_u holds the exact values of
// pd(x,i) - pd(x,u) at the four tet corners (|F| < 2^47) and C is the cofactor
// vector of at most three such rows (|C_c| < 6 * 2^141).  The dot product is
// below 2^192, so 256 bits (eight 32-bit limbs, two's complement) are exact.
#pragma once

#include <stdint.h>

struct I256 {
    uint32_t w[8];
};

__device__ __forceinline__ I256 i256_from_i128(__int128 v) {
    I256 r;
    unsigned __int128 u = (unsigned __int128)v;
#pragma unroll
    for (int k = 0; k < 4; k++) r.w[k] = (uint32_t)(u >> (32 * k));
    uint32_t s = v < 0 ? 0xffffffffu : 0u;
#pragma unroll
    for (int k = 4; k < 8; k++) r.w[k] = s;
    return r;
}

__device__ __forceinline__ I256 i256_add(const I256& a, const I256& b) {
    I256 r;
    uint64_t c = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        c += (uint64_t)a.w[k] + b.w[k];
        r.w[k] = (uint32_t)c;
        c >>= 32;
    }
    return r;
}

__device__ __forceinline__ I256 i256_neg(const I256& a) {
    I256 r;
    uint64_t c = 1;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        c += (uint64_t)(~a.w[k]);
        r.w[k] = (uint32_t)c;
        c >>= 32;
    }
    return r;
}

__device__ __forceinline__ bool i256_isneg(const I256& a) { return (a.w[7] >> 31) != 0; }

__device__ __forceinline__ int i256_sign(const I256& a) {
    if (i256_isneg(a)) return -1;
    uint32_t o = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) o |= a.w[k];
    return o ? 1 : 0;
}

// a * b for a 256-bit a and a signed 64-bit b (result must fit in 256 bits).
__device__ __forceinline__ I256 i256_mul_i64(I256 a, long long b) {
    bool neg = i256_isneg(a);
    if (neg) a = i256_neg(a);
    unsigned long long ub = b < 0 ? (unsigned long long)(-(b + 1)) + 1ull : (unsigned long long)b;
    if (b < 0) neg = !neg;
    uint32_t b0 = (uint32_t)ub, b1 = (uint32_t)(ub >> 32);
    I256 r;
    uint64_t carry = 0;
    // r = a*b0
#pragma unroll
    for (int k = 0; k < 8; k++) {
        uint64_t t = (uint64_t)a.w[k] * b0 + carry;
        r.w[k] = (uint32_t)t;
        carry = t >> 32;
    }
    // r += (a*b1) << 32
    carry = 0;
#pragma unroll
    for (int k = 1; k < 8; k++) {
        uint64_t t = (uint64_t)a.w[k - 1] * b1 + r.w[k] + carry;
        r.w[k] = (uint32_t)t;
        carry = t >> 32;
    }
    return neg ? i256_neg(r) : r;
}

__device__ __forceinline__ I256 i256_mul128_64(__int128 a, long long b) {
    return i256_mul_i64(i256_from_i128(a), b);
}

// Exact cofactor vector of m (1..3) rows R[0..m-1] over the m+1 free columns
// fc[0..m]: C_k = (-1)^k det(R without column k).  Rows hold values < 2^47.
__device__ inline void exact_cofactors(int m, const long long (*R)[4], const int* fc, I256* C) {
    if (m == 1) {
        C[0] = i256_from_i128((__int128)R[0][fc[1]]);
        C[1] = i256_from_i128(-(__int128)R[0][fc[0]]);
    } else if (m == 2) {
        long long x0 = R[0][fc[0]], x1 = R[0][fc[1]], x2 = R[0][fc[2]];
        long long y0 = R[1][fc[0]], y1 = R[1][fc[1]], y2 = R[1][fc[2]];
        C[0] = i256_from_i128((__int128)x1 * y2 - (__int128)x2 * y1);
        C[1] = i256_from_i128((__int128)x2 * y0 - (__int128)x0 * y2);
        C[2] = i256_from_i128((__int128)x0 * y1 - (__int128)x1 * y0);
    } else {
        for (int k = 0; k < 4; k++) {
            int c[3], n = 0;
            for (int q = 0; q < 4; q++)
                if (q != k) c[n++] = fc[q];
            // det3 of rows 0..2 on columns c
            __int128 m0 = (__int128)R[1][c[1]] * R[2][c[2]] - (__int128)R[1][c[2]] * R[2][c[1]];
            __int128 m1 = (__int128)R[1][c[0]] * R[2][c[2]] - (__int128)R[1][c[2]] * R[2][c[0]];
            __int128 m2 = (__int128)R[1][c[0]] * R[2][c[1]] - (__int128)R[1][c[1]] * R[2][c[0]];
            I256 d = i256_mul128_64(m0, R[0][c[0]]);
            d = i256_add(d, i256_neg(i256_mul128_64(m1, R[0][c[1]])));
            d = i256_add(d, i256_mul128_64(m2, R[0][c[2]]));
            C[k] = (k & 1) ? i256_neg(d) : d;
        }
    }
}
