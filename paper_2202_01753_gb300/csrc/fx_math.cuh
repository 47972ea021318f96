// fx_math.cuh -- natural logarithm and exponential of doubles whose range
// reduction and polynomial run in 64-bit fixed-point integer arithmetic.
//
// GB300 executes 2 FP64 fused multiply-adds per clock per SM against 64+
// integer multiply-adds, and the double-precision integrands spend most of
// their FP64 work in log and exp.  These versions follow P. T. P. Tang's
// table-driven methods ("Table-driven implementation of the logarithm
// function in IEEE floating-point arithmetic", ACM TOMS 16(4), 1990; "...of
// the exponential function...", ACM TOMS 15(2), 1989) with 256-entry tables
// (fx_tables.h, generated by gen_fx_tables.py), but evaluate the reduced
// argument's series in Q62 integers: the logarithm uses no FP64 operation
// (its parts are summed as a 128-bit fixed-point number and rounded to a
// double with integer operations), the exponential one (the FMA that picks
// n = round(y 256/ln 2); r = y - n ln2/256 is formed in 128-bit integers).
//
// Accuracy (tested against 60-digit references): fx_exp within 1 ulp;
// fx_log within 1 ulp plus 2^-58 absolute (the series is absolute-accurate,
// so for x within ~1e-3 of 1 the relative error grows as 2^-58 / |ln x|;
// every use in this library feeds an exponent or a difference, where the
// absolute error is what matters).  Outside the fast ranges (non-positive,
// subnormal, infinite or NaN x; |y| beyond ~708) they return CUDA's log/exp.
#pragma once

#include <cstdint>

#include "fx_tables.h"

namespace mc {
namespace fx {

// floor(a * b / 2^62) for signed Q62 operands, |a| < 2^61: one high multiply.
__device__ __forceinline__ int64_t mul_q62(int64_t a, int64_t b) { return __mul64hi(a * 4, b); }

constexpr int64_t kQ62One = (int64_t)1 << 62;

// Rounds the signed Q64 number v (value v / 2^64, |v| >= 1) to the nearest
// double (ties away from zero) using integer operations only.
__device__ __forceinline__ double q64_to_double(__int128 v)
{
    const bool neg = v < 0;
    unsigned __int128 a = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
    const uint64_t hw = (uint64_t)(a >> 64);
    const int p = hw ? 127 - __clzll((long long)hw) : 63 - __clzll((long long)(uint64_t)a);  // leading bit
    uint64_t m;
    int e = p - 64 + 1023;
    if (p > 52) {
        const int sh = p - 52;
        m = (uint64_t)((a + ((unsigned __int128)1 << (sh - 1))) >> sh);
        if (m >> 53) {  // rounding carried into a new leading bit
            m >>= 1;
            ++e;
        }
    } else {
        m = (uint64_t)a << (52 - p);
    }
    const uint64_t bits = ((uint64_t)neg << 63) | ((uint64_t)e << 52) | (m & 0xFFFFFFFFFFFFFull);
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ double fx_log(double x)
{
    const uint64_t u = (uint64_t)__double_as_longlong(x);
    if (u - 0x0010000000000000ull >= 0x7FE0000000000000ull) return log(x);  // not a positive normal number
    const int e = (int)(u >> 52) - 1023;
    const uint64_t f = u & 0xFFFFFFFFFFFFFull;
    const int j = (int)(f >> 44);  // nearest table point c_j = 1 + (j + 1/2)/256
    // m - c_j in Q52 (|.| <= 2^43), then r = (m - c_j) / c_j in Q62 (|r| <= 2^-9)
    const int64_t D = (int64_t)f - ((int64_t)(2 * j + 1) << 43);
    const int64_t r = __mul64hi((int64_t)((uint64_t)D << 11), (int64_t)__ldg(&kLogInvC[j]));
    // ln(1 + r) = r - r^2/2 + r^3/3 - r^4/4 + r^5/5 - r^6/6 (+ |r|^7/7 < 2^-65)
    int64_t s = -kQ62One / 6;
    s = kQ62One / 5 + mul_q62(r, s);
    s = -kQ62One / 4 + mul_q62(r, s);
    s = kQ62One / 3 + mul_q62(r, s);
    s = -kQ62One / 2 + mul_q62(r, s);
    s = kQ62One + mul_q62(r, s);
    const int64_t l1 = mul_q62(r, s);
    // ln x = e ln2 + ln c_j + ln(1 + r), summed as a Q64 fixed-point number
    const __int128 v = (__int128)e * (__int128)kLn2W1 + (((__int128)e * (__int128)kLn2W2) >> 64) +
                       (__int128)__ldg(&kLogCQ64[j]) + ((__int128)l1 << 2);
    if (v == 0) return 0.0;
    return q64_to_double(v);
}

__device__ __forceinline__ double fx_exp(double y)
{
    const uint64_t u = (uint64_t)__double_as_longlong(y);
    const uint64_t ay = u & 0x7FFFFFFFFFFFFFFFull;
    if (ay >= 0x4086200000000000ull) return exp(y);  // |y| >= 708 (or NaN): CUDA's exp
    if (ay < 0x3C30000000000000ull) return 1.0 + y;  // |y| < 2^-60: exp(y) rounds from 1 + y
    // y = n ln2/256 + r, n = round(y 256/ln2) by the 1.5 * 2^52 shift (one FMA)
    const double t = fma(y, k256OverLn2, 0x1.8p52);
    const int64_t n = __double_as_longlong(t) - __double_as_longlong(0x1.8p52);
    // r = y - n ln2/256 in Q62 with integers: y exactly (bits below 2^-62
    // dropped; |y| < 2^10 fits 72 bits) minus n ln2/256 from a Q115 constant
    const int sh = (int)((u >> 52) & 0x7FF) - 1013;  // y = M 2^(E-1075): Q62 needs a shift by E - 1013
    const uint64_t M = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    __int128 Y = sh >= 0 ? ((__int128)M << sh) : (__int128)(M >> -sh);
    if (u >> 63) Y = -Y;
    const __int128 C = ((__int128)kLn2Over256Q115Hi << 64) | (__int128)kLn2Over256Q115Lo;
    const __int128 L = ((__int128)n * C + ((__int128)1 << 52)) >> 53;
    const int64_t rq = (int64_t)(Y - L);  // |r| <= ln2/512 + tiny: |rq| < 2^54
    // e^r = 1 + r + r^2/2 + r^3/6 + r^4/24 + r^5/120 (+ |r|^6/720 < 2^-66)
    int64_t s = kQ62One / 120;
    s = kQ62One / 24 + mul_q62(rq, s);
    s = kQ62One / 6 + mul_q62(rq, s);
    s = kQ62One / 2 + mul_q62(rq, s);
    s = kQ62One + mul_q62(rq, s);
    s = kQ62One + mul_q62(rq, s);
    // 2^(j/256) e^r in Q62, within [0.9986, 2)
    const int j = (int)(n & 255);
    const int k = (int)(n >> 8);
    const uint64_t P = __umul64hi(__ldg(&kExp2[j]) << 1, (uint64_t)s << 1);
    // assemble 2^k P / 2^62 (rounded to nearest, ties away), a normal double for |y| < 708
    uint64_t bits;
    if (P >= ((uint64_t)1 << 62))
        bits = ((uint64_t)(k + 1023) << 52) + (((P + (1ull << 9)) >> 10) - (1ull << 52));
    else
        bits = ((uint64_t)(k + 1022) << 52) + (((P + (1ull << 8)) >> 9) - (1ull << 52));
    return __longlong_as_double((long long)bits);
}

// Single-precision cosine for the mixed-precision kernels: x = k pi/2 + r
// with k = rint(x 2/pi) and r = x - k pi/2 by a three-term Cody-Waite
// reduction with fused multiply-adds (pi/2 = F1 + F2 + F3; the products are
// exact inside the FMAs), |r| <= pi/4 (plus rounding); then cos x = cos r,
// -sin r, -cos r or sin r by k mod 4, with the Taylor series
// cos r = 1 - r^2/2! + ... + r^8/8! (next term < 2.5e-8) and
// sin r = r - r^3/3! + ... + r^9/9! (next term < 2.2e-9).  Error: a few
// units of 2^-24 for |x| < 2^22 (tested against CUDA's cosf).  Beyond 2^22,
// where a float argument is itself known only to about 0.5, the hardware
// approximation __cosf is used; no local-memory slow path is compiled in.
__device__ __forceinline__ float fx_cosf(float x)
{
    if (!(fabsf(x) < 4194304.0f)) return __cosf(x);
    const float k = rintf(x * kTwoOverPiF);
    float r = fmaf(-k, kHalfPiF1, x);
    r = fmaf(-k, kHalfPiF2, r);
    r = fmaf(-k, kHalfPiF3, r);
    const float r2 = r * r;
    float c = 1.0f / 40320.0f;
    c = fmaf(c, r2, -1.0f / 720.0f);
    c = fmaf(c, r2, 1.0f / 24.0f);
    c = fmaf(c, r2, -0.5f);
    c = fmaf(c, r2, 1.0f);
    float s = 1.0f / 362880.0f;
    s = fmaf(s, r2, -1.0f / 5040.0f);
    s = fmaf(s, r2, 1.0f / 120.0f);
    s = fmaf(s, r2, -1.0f / 6.0f);
    s = fmaf(s * r2, r, r);
    const int q = (int)k & 3;
    const float v = (q & 1) ? s : c;
    return (q == 1 || q == 2) ? -v : v;
}

}  // namespace fx
}  // namespace mc
