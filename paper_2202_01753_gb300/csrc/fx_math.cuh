// fx_math.cuh -- natural logarithm and exponential of doubles whose range
// reduction and polynomial run in 64-bit fixed-point integer arithmetic.
//
// GB300 executes 2 FP64 fused multiply-adds per clock per SM against 64+
// integer multiply-adds, and the double-precision integrands spend most of
// their FP64 work in log and exp.  These versions follow P. T. P. Tang's
// table-driven methods ("Table-driven implementation of the logarithm
// function in IEEE floating-point arithmetic", ACM TOMS 16(4), 1990; "...of
// the exponential function...", ACM TOMS 15(2), 1989) with 256-entry tables
// (fx_tables.h, generated by gen_fx_tables.py), applied twice -- a second
// 256-entry table step takes the reduced argument from below 2^-8 to below
// 2^-16, so that three series terms, formed with 32-bit multiplies, replace
// seven and the long chain of dependent 64-bit multiplies -- and evaluate
// everything in fixed-point integers: the logarithm uses no FP64 operation
// (its table points are the ones at or below the argument, so every quantity
// is non-negative; its parts are summed as a 128-bit fixed-point number and
// rounded to a double with integer operations), the exponential none either
// (n = round(y 256/ln 2) from y's significand by one high multiply;
// r = y - n ln2/256 is formed from the low 64 bits of its two terms and made
// non-negative).  fx_exp_neg_scaled multiplies the result by a 64-bit
// fixed-point factor before its single rounding (the FP64 kernels' Jacobian,
// kept as an integer product), which saves the FP64 multiply after it.
//
// Accuracy (tested against 60-digit references): fx_exp within 1 ulp
// (subnormal results within one unit of their last place);
// fx_log within 1 ulp plus 2^-58 absolute (the series is absolute-accurate,
// so for x within ~1e-3 of 1 the relative error grows as 2^-58 / |ln x|;
// every use in this library feeds an exponent or a difference, where the
// absolute error is what matters).  Outside the fast ranges (non-positive,
// subnormal, infinite or NaN x; y above ~708) they return CUDA's log/exp.
#pragma once

#include <cstdint>

#include "fx_tables.h"

namespace mc {
namespace fx {

// Rounds (-1)^neg (hi 2^64 + lo) / 2^64, a nonzero magnitude below 2^10
// (hi < 2^10), to a double (ties away from zero) with 64-bit integer
// operations: a value >= 1 from its Q54 window hi 2^54 + lo 2^-10 (the
// dropped bits are below a quarter of its last place), a value < 1 from lo.
__device__ __forceinline__ double q64_to_double(uint64_t hi, uint64_t lo, bool neg)
{
    const bool big = hi != 0;
    const uint64_t t = big ? ((hi << 54) | (lo >> 10)) : lo;
    const int p = 63 - __clzll((long long)t);  // leading bit of t
    int e = p - (big ? 54 : 64) + 1023;
    uint64_t m;
    if (p > 52) {
        const int sh = p - 52;
        m = (t >> sh) + ((t >> (sh - 1)) & 1ull);
        if (m >> 53) {  // rounding carried into a new leading bit
            m >>= 1;
            ++e;
        }
    } else {
        m = t << (52 - p);
    }
    const uint64_t bits = ((uint64_t)neg << 63) | (((uint64_t)e << 52) + m - (1ull << 52));
    return __longlong_as_double((long long)bits);
}

// The rare cases go to CUDA's functions through calls, so that their code is
// not inlined into every use (the sampling loop inlines the fast paths once
// per axis; inlined slow paths multiply its size and its instruction-fetch
// stalls).
static __device__ __noinline__ double log_slow(double x) { return log(x); }
static __device__ __noinline__ double exp_slow(double y) { return exp(y); }

// Constant of the series: round(2^32 / k).
__host__ __device__ constexpr uint32_t q32_inv(uint32_t k) { return (uint32_t)((((uint64_t)1 << 32) + k / 2) / k); }

// A logarithm table entry, one 16-byte load through the read-only cache.
__device__ __forceinline__ LogPair ld_pair(const LogPair* p)
{
#ifdef __CUDA_ARCH__
    const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(p));
    return LogPair{v.x, v.y};
#else
    return *p;
#endif
}

// ln x = e ln 2 + ln c_j + ln d_k + ln(1 + r2) for x = 2^e m, c_j = 1 + j/256
// the table point at or below m, r = (m - c_j)/c_j in [0, 2^-8), d_k =
// 1 + k/65536 the second table point at or below 1 + r and r2 = (r - k/65536)/d_k
// in [0, 2^-16): every quantity is non-negative.
__device__ __forceinline__ double fx_log(double x)
{
    const uint64_t u = (uint64_t)__double_as_longlong(x);
    if ((uint32_t)(u >> 32) - 0x00100000u >= 0x7FE00000u) return log_slow(x);  // not a positive normal number
    const int e = (int)(u >> 52) - 1023;
    const uint64_t f = u & 0xFFFFFFFFFFFFFull;
    const int j = (int)(f >> 44);
    // m - c_j is the mantissa's low 44 bits (Q52); r = (m - c_j)/c_j in Q64 (< 2^56)
    const LogPair cj = ld_pair(&kLogC[j]);
    const uint64_t r = __umul64hi((f & 0xFFFFFFFFFFFull) << 13, cj.inv);
    // second step: k = the top 8 bits of r (r < 2^-8), r - k/65536 its low 48 bits
    // (Q64); r2 = (r - k/65536)/d_k in Q64 (< 2^48)
    const int k = (int)(r >> 48);
    const LogPair dk = ld_pair(&kLogD[k]);
    const uint64_t R = __umul64hi((r & 0xFFFFFFFFFFFFull) << 16, dk.inv) >> 15;
    // ln(1 + r2) = r2 - r2^2/2 + r2^3/3 (+ r2^4/4 < 2^-66).  r2^2 from the top 32
    // bits of r2 (H = r2 in Q48; the dropped low bits move it by < 2^-62) and
    // r2^3 < 2^-48 from r2^2 and H, both with 32 x 32-bit products.
    const uint32_t H = (uint32_t)(R >> 16);
    const uint64_t sq = ((uint64_t)H * H) >> 32;                           // r2^2, Q64 (< 2^32)
    const uint32_t cube = (uint32_t)(((uint64_t)(uint32_t)sq * H) >> 48);  // r2^3, Q64 (< 2^16)
    const uint64_t l2 = R - (sq >> 1) + __umulhi(cube, q32_inv(3));        // ln(1 + r2), Q64
    const uint64_t U = cj.ln + dk.ln + l2;                                 // ln m, Q64 (< ln 2)
    // e ln 2 + ln m as sign and 128-bit magnitude in Q64; |e| < 2^11, so
    // |e| ln 2 is two 32 x 32-bit products (ln 2 = L1 2^32 + L0)
    const uint32_t ae = (uint32_t)(e < 0 ? -e : e);
    const uint64_t p0 = (uint64_t)ae * (uint32_t)kLn2Q64;
    const uint64_t p1 = (uint64_t)ae * (uint32_t)(kLn2Q64 >> 32);
    const uint64_t plo = p0 + (p1 << 32);
    const uint64_t phi = (p1 >> 32) + (plo < p0 ? 1ull : 0ull);
    uint64_t lo, hi;
    bool neg = false;
    if (e >= 0) {
        lo = plo + U;
        hi = phi + (lo < U ? 1ull : 0ull);
    } else {
        lo = plo - U;
        hi = phi - (plo < U ? 1ull : 0ull);
        neg = true;
        if ((int64_t)hi < 0) {  // ln m > |e| ln 2 by rounding (x just below 1): a tiny positive value
            lo = 0ull - lo;
            hi = ~hi + (lo == 0 ? 1ull : 0ull);
            neg = false;
        }
    }
    if ((hi | lo) == 0) return 0.0;
    return q64_to_double(hi, lo, neg);
}

// exp of the double with bits u; SCALED: exp(y) (jm / 2^63) 2^je, jm in
// [2^63, 2^64), rounded once.  The scaled form keeps the unscaled one's
// special cases: where exp(y) alone rounds to +0 the result is +0 (as
// exp(y) * J would be), and exp(y)'s subnormal range is scaled exactly.
template <bool SCALED>
__device__ __forceinline__ double fx_exp_bits_t(uint64_t u, uint64_t jm, int je)
{
    const double y = __longlong_as_double((long long)u);
    const uint64_t ay = u & 0x7FFFFFFFFFFFFFFFull;
    const uint32_t ayh = (uint32_t)(ay >> 32);  // the thresholds below have zero low words
    if (ayh >= 0x40862000u) {  // |y| >= 708, infinite or NaN
        // y < -745.2 (down to -inf): exp(y) < 2^-1075 rounds to +0.  Integrands
        // with narrow peaks land here often, so it takes no FP64 work.  Down
        // from -708 the results are subnormal; they are assembled below with
        // integer rounding, so that these samples (a few percent of a narrow
        // peak's) do not send their warp through CUDA's exp with one or two
        // lanes on the FP64 pipe.  Overflow and NaN are CUDA's exp.
        if (!(u >> 63) || ay > 0x7FF0000000000000ull) {
            if constexpr (SCALED) return exp_slow(y) * ldexp((double)jm, je - 63);
            else return exp_slow(y);
        }
        if (ay > 0x408749999999999Aull) return 0.0;
    }
    if (ayh < 0x3C300000u) {  // |y| < 2^-60: exp(y) rounds to 1
        if constexpr (SCALED) return ldexp((double)jm, je - 63);
        else return 1.0;
    }
    // y = n ln2/256 + r, n = round(y 256/ln2) from y's significand M and
    // exponent E: |y| 256/ln2 = H 2^(E-1075) to 2^-52 relative, H =
    // floor(M K / 2^53) with K = 256/ln2 in Q53, rounded at bit 1075 - E (>= 43).
    // Near a tie n may be the other neighbour: |r| stays below ln2/256.
    const int E = (int)((u >> 52) & 0x7FF);
    const uint64_t M = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const uint64_t H = __umul64hi(M << 11, k256OverLn2Q53);
    const int sh1 = 1074 - E;  // the rounding bit's position minus one
    const int64_t na = (int64_t)(((sh1 < 64 ? H >> sh1 : 0ull) + 1ull) >> 1);
    int64_t n = (u >> 63) ? -na : na;
    // r = y - n ln2/256 in Q62 (|r| <= ln2/512 + tiny: |rq| < 2^54), so only the
    // low 64 bits of y in Q62 and of n ln2/256 matter: y's bits below 2^-62 are
    // dropped; n ln2/256 = (n C + 2^52) >> 53 with C = ln2/256 in Q115 =
    // Hi 2^64 + Lo, of which bits 53..116 are kept
    const int sh = E - 1013;  // y = M 2^(E-1075): Q62 needs a shift by E - 1013
    uint64_t Y = sh >= 0 ? M << sh : (sh > -64 ? M >> -sh : 0ull);
    if (u >> 63) Y = 0ull - Y;
    const uint64_t nu = (uint64_t)n;
    const uint64_t plo = nu * kLn2Over256Q115Lo;
    uint64_t phi = __umul64hi(nu, kLn2Over256Q115Lo) - (n < 0 ? kLn2Over256Q115Lo : 0ull);  // n Lo, signed
    const uint64_t plo2 = plo + (1ull << 52);
    phi += plo2 < plo ? 1ull : 0ull;
    const uint64_t L = ((phi + nu * kLn2Over256Q115Hi) << 11) | (plo2 >> 53);
    int64_t rq = (int64_t)(Y - L);
    if (rq < 0) {  // r in [0, ln2/256): n one lower
        --n;
        rq += (int64_t)kLn2Over256Q62;
    }
    // e^r = e^(q/65536) e^b with q = floor(r 65536) (< 178) and b < 2^-16 (Q62 < 2^46):
    // e^b = 1 + b + b^2/2 + b^3/6 (+ b^4/24 < 2^-68), b^2 from the top 32 bits of b
    // (Hb = b in Q48) and b^3 from b^2 and Hb, with 32 x 32-bit products
    const uint32_t q = (uint32_t)((uint64_t)rq >> 46);
    const uint64_t B = (uint64_t)rq & ((1ull << 46) - 1);
    const uint32_t Hb = (uint32_t)(B >> 14);
    const uint64_t sqb = ((uint64_t)Hb * Hb) >> 34;                      // b^2 in Q62 (< 2^30)
    const uint32_t cub = (uint32_t)((sqb * Hb) >> 48);                   // b^3 in Q62 (< 2^14)
    const uint64_t eb = (1ull << 62) + B + (sqb >> 1) + __umulhi(cub, q32_inv(6));  // e^b, Q62
    const uint64_t s = __umul64hi(__ldg(&kExpK16[q]) << 1, eb << 1);     // e^r, Q62
    // 2^(j/256) e^r in Q62, within [1, 2)
    const int j = (int)(n & 255);
    const int k = (int)(n >> 8);
    const uint64_t P = __umul64hi(__ldg(&kExp2[j]) << 1, s << 1);
    // assemble 2^k P / 2^62 (rounded to nearest, ties away): P normalised
    // into [2^62, 2^63), then a normal double (biased exponent eb >= 1) or,
    // for eb <= 0 (y below about -708.4), the subnormal round(P 2^-(11 - eb))
    // (a carry into 2^52 is the smallest normal; below 2^-1075 it is +0)
    uint64_t Pn = P;
    int be = k + 1023;  // biased exponent
    if constexpr (SCALED) {
        Pn = __umul64hi(P << 1, jm);  // Q62, a value in [1, 4)
        be += je;
        if (Pn >> 63) {
            Pn >>= 1;
            ++be;
        }
        if (be >= 2047) return __longlong_as_double(0x7FF0000000000000ll);  // overflow: +inf
    }
    if (Pn < ((uint64_t)1 << 62)) {
        Pn <<= 1;
        --be;
    }
    uint64_t bits;
    if (be >= 1) {
        bits = ((uint64_t)be << 52) + (((Pn + (1ull << 9)) >> 10) - (1ull << 52));
    } else {
        const int sh = 11 - be;
        bits = sh < 64 ? (Pn + (1ull << (sh - 1))) >> sh : 0ull;
    }
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ double fx_exp_bits(uint64_t u) { return fx_exp_bits_t<false>(u, 0, 0); }

__device__ __forceinline__ double fx_exp(double y) { return fx_exp_bits((uint64_t)__double_as_longlong(y)); }

// exp(-v) (jm / 2^63) 2^je (jm in [2^63, 2^64)), rounded once
__device__ __forceinline__ double fx_exp_neg_scaled(double v, uint64_t jm, int je)
{
    return fx_exp_bits_t<true>((uint64_t)__double_as_longlong(v) ^ 0x8000000000000000ull, jm, je);
}

// exp(-v), the sign flipped on the bits (no FP64 negation)
__device__ __forceinline__ double fx_exp_neg(double v)
{
    return fx_exp_bits((uint64_t)__double_as_longlong(v) ^ 0x8000000000000000ull);
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
