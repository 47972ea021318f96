// mc_device.cuh -- device building blocks of the sampling kernel:
// counter-based random words, the exact sub-cube/bin position of a
// coordinate, the integrand families, and compensated single-precision sums.
#pragma once

#include <cstdint>

#include "fx_math.cuh"
#include "mc_internal.h"

namespace mc {

// ---------------------------------------------------------------------------
// Double-double arithmetic (value = hi + lo, |lo| <= ulp(hi)/2): error-free
// TwoSum (Knuth) and an FMA-based exact product (Dekker).  Grid edges are held
// in this form so that a narrow bin's width (a difference of two nearly equal
// edges, and a factor of the Jacobian) keeps full relative precision; the
// rebinning forms each new edge (left + width * fraction) in it.
// ---------------------------------------------------------------------------
struct DD {
    double hi, lo;
};

__device__ __forceinline__ DD dd_two_sum(double a, double b)
{
    const double s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    return DD{s, __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb))};
}

__device__ __forceinline__ DD dd_renorm(double hi, double lo)
{
    const double s = __dadd_rn(hi, lo);
    return DD{s, __dsub_rn(lo, __dsub_rn(s, hi))};
}

__device__ __forceinline__ DD dd_add(DD a, DD b)
{
    const DD t = dd_two_sum(a.hi, b.hi);
    return dd_renorm(t.hi, __dadd_rn(__dadd_rn(t.lo, a.lo), b.lo));
}

__device__ __forceinline__ DD dd_scale(DD a, double b)
{
    const double p = __dmul_rn(a.hi, b);
    const double e = __fma_rn(a.hi, b, -p);
    return dd_renorm(p, __fma_rn(a.lo, b, e));
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11).  The round keys (key + r * Weyl increments) are
// precomputed on the host and read from the kernel's constant bank.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 x, const uint32_t (&rk)[10][2])
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t a0 = x.x * 0xD2511F53u, h0 = __umulhi(x.x, 0xD2511F53u);
        const uint32_t a1 = x.z * 0xCD9E8D57u, h1 = __umulhi(x.z, 0xCD9E8D57u);
        x = make_uint4(h1 ^ x.y ^ rk[r][0], a1, h0 ^ x.w ^ rk[r][1], a0);
    }
    return x;
}

// The same generator with the round keys formed on the fly from the key
// (for kernels whose key is per-integral data rather than a launch constant).
__device__ __forceinline__ uint4 philox4x32_10_key(uint4 x, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t a0 = x.x * 0xD2511F53u, h0 = __umulhi(x.x, 0xD2511F53u);
        const uint32_t a1 = x.z * 0xCD9E8D57u, h1 = __umulhi(x.z, 0xCD9E8D57u);
        x = make_uint4(h1 ^ x.y ^ k0, a1, h0 ^ x.w ^ k1, a0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return x;
}

__device__ __forceinline__ uint4 sample_words(const VsArgs& a, uint4 ctr) { return philox4x32_10(ctr, a.rk); }

// Register view of one batch integral for the per-sample code (the family
// constants stay in shared memory).
struct BatchView {
    uint32_t d, nb, g, gmagic, key0, key1;
    uint32_t hist_d;  // axes with a histogram (d)
    double jac0;
    float phi_scale_f;
    double inv_p, inv_var_den;     // 1/p, 1/(p (p-1))
    float inv_p_f, inv_var_den_f;
    uint32_t want_abs;             // 0: a batch iteration does not use the sums of |cube mean|
    const FamParams& fam;
};

__device__ __forceinline__ uint4 sample_words(const BatchView& v, uint4 ctr)
{
    return philox4x32_10_key(ctr, v.key0, v.key1);
}

// ---------------------------------------------------------------------------
// Product of positive doubles in integer arithmetic (the FP64 kernels'
// Jacobian): the running value is m 2^(e - 63) with m in [2^63, 2^64); each
// factor's 53-bit significand is multiplied in as a 64 x 64 -> high-64
// product (truncated: < 2^-63 relative per factor) and renormalised by one
// bit; the result is rounded to a double once.  No FP64 instruction (GB300
// issues 2 per clock per SM, the integer multiplies run elsewhere).
// ---------------------------------------------------------------------------
struct IntProd {
    uint64_t m;
    int e;
};

__device__ __forceinline__ IntProd int_prod_of(double v)  // v > 0, finite
{
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    const int E = (int)(b >> 52);
    const uint64_t mant = b & 0xFFFFFFFFFFFFFull;
    if (E) return IntProd{(mant | (1ull << 52)) << 11, E - 1023};
    const int s = __clzll((long long)mant);  // subnormal
    return IntProd{mant << s, -1074 + 63 - s};
}

__device__ __forceinline__ void int_prod_mul(IntProd& p, double v)
{
    const IntProd f = int_prod_of(v);
    const uint64_t H = __umul64hi(p.m, f.m);
    const uint64_t top = H >> 63;
    p.m = top ? H : H << 1;
    p.e += f.e + (int)top;
}

__device__ __forceinline__ double int_prod_value(const IntProd& p)
{
    // rounded to 53 bits (2^53 after a carry); m + 2^10 could wrap around
    const uint64_t r = (p.m >> 11) + ((p.m >> 10) & 1ull);
    const int E = p.e + 1023;
    if (E < 1 || E > 2046) return ldexp((double)r, p.e - 52);  // beyond the normal range: rare
    return __longlong_as_double((long long)(((uint64_t)E << 52) + r - (1ull << 52)));
}

// ---------------------------------------------------------------------------
// Map cell k of one axis in the box's coordinates, from the double-double
// right edges (unit cube) of that axis's row: (x left edge, x width / g) for
// the FP64 kernels, (x left edge, nb * x width) in single precision for the
// mixed ones.  inv_g = 1 / g.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void map_cell_edges(DD left, DD right, double lo, double scale, double* xl, double* xw)
{
    const DD wd = dd_add(right, DD{-left.hi, -left.lo});
    *xl = lo + scale * left.hi;
    *xw = scale * (wd.hi + wd.lo);
}

__device__ __forceinline__ void map_cell(const double* row, const double* row_lo, uint32_t k, double lo,
                                         double scale, double* xl, double* xw)
{
    const DD right{row[k], row_lo[k]};
    const DD left = k ? DD{row[k - 1], row_lo[k - 1]} : DD{0.0, 0.0};
    map_cell_edges(left, right, lo, scale, xl, xw);
}

__device__ __forceinline__ double2 map_cell_f64(const double* row, const double* row_lo, uint32_t k, double lo,
                                                double scale, double inv_g)
{
    double xl, xw;
    map_cell(row, row_lo, k, lo, scale, &xl, &xw);
    return make_double2(xl, xw * inv_g);
}

__device__ __forceinline__ float2 map_cell_f32(const double* row, const double* row_lo, uint32_t k, double lo,
                                               double scale, uint32_t nb)
{
    double xl, xw;
    map_cell(row, row_lo, k, lo, scale, &xl, &xw);
    return make_float2((float)xl, (float)(xw * (double)nb));
}

// ---------------------------------------------------------------------------
// Exact position of one coordinate (Alg. 1 map step, Alg. 3 Get-Bin-ID).  The
// sample sits at y = (c + u)/g on this axis, c the sub-cube digit and
// u = (w + 1/2) / 2^32 the offset drawn from the random word w.  With
// A = nb (2w + 1) = a_hi 2^33 + a_lo and Q = nb c + a_hi:
//     nb y = (Q + a_lo 2^-33) / g,   k = floor(Q / g),
//     phi = nb y - k = (Q mod g + a_lo 2^-33) / g.
// Q < nb g <= 2^31, so floor(Q/g) is one high multiply by
// gmagic = floor((2^32-1)/g) and at most one correction.
// ---------------------------------------------------------------------------
struct BinPos {
    uint32_t k;    // bin index
    uint32_t r;    // Q mod g
    uint32_t ahi;  // bit 32 of a_lo (i.e. A >> 32 & 1)
    uint32_t alo;  // low 32 bits of a_lo
};

__device__ __forceinline__ BinPos bin_pos(uint32_t w, uint32_t nb_c, uint32_t nb, uint32_t g,
                                          uint32_t gmagic)
{
    const uint64_t A = (uint64_t)(2u * nb) * (uint64_t)w + (uint64_t)nb;
    const uint32_t hi = (uint32_t)(A >> 32);
    const uint32_t Q = nb_c + (hi >> 1);
    uint32_t q = __umulhi(Q, gmagic);
    uint32_t r = Q - q * g;
    if (r >= g) { ++q; r -= g; }
    BinPos b;
    b.k = q;
    b.r = r;
    b.ahi = hi & 1u;
    b.alo = (uint32_t)A;
    return b;
}

// g phi = r + a_lo 2^-33 as a double, built from the integer numerator
// r 2^33 + a_lo with integer operations only (exact below 2^53, rounded to
// nearest above): no FP64 conversion or multiply in the sampling loop.  The
// numerator is never 0: its low 33 bits are those of A = nb (2w + 1), an odd
// multiple of nb < 2^33.
__device__ __forceinline__ double bin_gphi_f64(const BinPos& b)
{
    const uint64_t num = ((uint64_t)b.r << 33) | ((uint64_t)b.ahi << 32) | (uint64_t)b.alo;  // < 2^63
    const int lz = __clzll((long long)num);
    uint64_t m;  // num with its leading one moved to bit 52 (bit 53 after a rounding carry)
    if (lz >= 11) {
        m = num << (lz - 11);
    } else {
        const int sh = 11 - lz;
        m = (num + (1ull << (sh - 1))) >> sh;
    }
    // value 2^(63 - lz - 33) (m / 2^52): biased exponent 1053 - lz, stored as
    // (exponent - 1) << 52 plus m, whose leading one adds the missing 1
    const uint64_t bits = ((uint64_t)(1052 - lz) << 52) + m;
    return __longlong_as_double((long long)bits);
}

// the same in single precision: (r + a_lo 2^-33) * scale, scale = 1/g for phi
__device__ __forceinline__ float bin_phi_f32(const BinPos& b, float scale)
{
    const float base = __uint2float_rn(b.r) + (b.ahi ? 0.5f : 0.0f);
    return __fmul_rn(__fmaf_rn(__uint2float_rn(b.alo), 1.16415321826934814453125e-10f /*2^-33*/, base), scale);
}

// ---------------------------------------------------------------------------
// Integrand families.  Each keeps a running state updated axis by axis, so
// the point x never has to be stored; constants come from FamParams, whose
// layout per family is fixed by integrand_prepare (capi.cu):
//   CONST    c[0] = v
//   GAUSS    c[0] = A, c[1+j] = mu_j, c[13+j] = 1/(2 sig_j^2)
//   CORNER   c[j] = a_j
//   OSC      c[0] = 2 pi u, c[1+j] = a_j
//   PRODPEAK c[j] = c_j^-2, c[12+j] = w_j
//   C0       c[j] = c_j, c[12+j] = w_j
//   DISCONT  c[j] = c_j, c[12+j] = w_j
//   COSMO6   c[0..5] = a (c[2], c[3] = a_3 + 1, a_4 + 1), c[6] = mu, c[7] = 1/(2 s^2), c[8] = r, c[9] = 1/(2 t^2),
//            c[10] = 1/(2 pi s^2) (FP64: in the Jacobian's constant), c[11], c[12] = c[2], c[3] - 2 c7 mu,
//            c[13] = 2 c7 mu^2
// ---------------------------------------------------------------------------
template <typename R> struct RealOps;
template <> struct RealOps<double> {
    // fixed-point table-driven versions: a few FP64 operations instead of tens
    __device__ static double exp_(double v) { return fx::fx_exp(v); }
    __device__ static double expm_(double v) { return fx::fx_exp_neg(v); }   // exp(-v)
    __device__ static double log_(double v) { return fx::fx_log(v); }
    __device__ static double cos_(double v) { return cos(v); }
    __device__ static double rcp(double v) { return 1.0 / v; }
    __device__ static double par(const FamParams& f, int i) { return f.c[i]; }
};
template <> struct RealOps<float> {
    __device__ static float exp_(float v) { return expf(v); }
    __device__ static float expm_(float v) { return expf(-v); }
    __device__ static float log_(float v) { return logf(v); }
    __device__ static float cos_(float v) { return fx::fx_cosf(v); }
    __device__ static float rcp(float v) { return 1.0f / v; }
    __device__ static float par(const FamParams& f, int i) { return f.cf[i]; }
};

template <int FAM, typename R> struct Family;

template <typename R> struct Family<MCUBES_F_CONST, R> {
    struct S {};
    __device__ static void begin(S&) {}
    __device__ static void add(S&, int, R, const FamParams&) {}
    __device__ static R end(const S&, uint32_t, const FamParams& f) { return RealOps<R>::par(f, 0); }
};

template <typename R> struct Family<MCUBES_F_GAUSS, R> {
    struct S { R q; };
    __device__ static void begin(S& s) { s.q = R(0); }
    __device__ static void add(S& s, int j, R x, const FamParams& f)
    {
        const R z = x - RealOps<R>::par(f, 1 + j);
        s.q += z * z * RealOps<R>::par(f, 13 + j);
    }
    __device__ static R end(const S& s, uint32_t, const FamParams& f)
    {
        return RealOps<R>::par(f, 0) * RealOps<R>::expm_(s.q);
    }
};

template <typename R> struct Family<MCUBES_F_CORNER, R> {
    struct S { R t; };
    __device__ static void begin(S& s) { s.t = R(1); }
    __device__ static void add(S& s, int j, R x, const FamParams& f) { s.t += RealOps<R>::par(f, j) * x; }
    __device__ static R end(const S& s, uint32_t d, const FamParams&)
    {
        // t^-(d+1) by repeated squaring of 1/t
        R b = RealOps<R>::rcp(s.t), r = R(1);
        uint32_t e = d + 1;
        while (e) {
            if (e & 1u) r *= b;
            b *= b;
            e >>= 1;
        }
        return r;
    }
};

template <typename R> struct Family<MCUBES_F_OSC, R> {
    struct S { R t; };
    __device__ static void begin(S& s) { s.t = R(0); }
    __device__ static void add(S& s, int j, R x, const FamParams& f) { s.t += RealOps<R>::par(f, 1 + j) * x; }
    __device__ static R end(const S& s, uint32_t, const FamParams& f)
    {
        return RealOps<R>::cos_(RealOps<R>::par(f, 0) + s.t);
    }
};

template <typename R> struct Family<MCUBES_F_PRODPEAK, R> {
    struct S { R v; };
    __device__ static void begin(S& s) { s.v = R(1); }
    __device__ static void add(S& s, int j, R x, const FamParams& f)
    {
        const R z = x - RealOps<R>::par(f, 12 + j);
        s.v *= RealOps<R>::rcp(RealOps<R>::par(f, j) + z * z);
    }
    __device__ static R end(const S& s, uint32_t, const FamParams&) { return s.v; }
};

template <typename R> struct Family<MCUBES_F_C0, R> {
    struct S { R t; };
    __device__ static void begin(S& s) { s.t = R(0); }
    __device__ static void add(S& s, int j, R x, const FamParams& f)
    {
        const R z = x - RealOps<R>::par(f, 12 + j);
        s.t += RealOps<R>::par(f, j) * (z < R(0) ? -z : z);
    }
    __device__ static R end(const S& s, uint32_t, const FamParams&) { return RealOps<R>::expm_(s.t); }
};

template <typename R> struct Family<MCUBES_F_DISCONT, R> {
    struct S { R t; bool out; };
    __device__ static void begin(S& s) { s.t = R(0); s.out = false; }
    __device__ static void add(S& s, int j, R x, const FamParams& f)
    {
        s.out |= !(x < RealOps<R>::par(f, 12 + j));
        s.t += RealOps<R>::par(f, j) * x;
    }
    __device__ static R end(const S& s, uint32_t, const FamParams&)
    {
        return s.out ? R(0) : RealOps<R>::exp_(s.t);
    }
};

template <typename R> struct Family<MCUBES_F_COSMO6, R> {
    // f = c10 exp(-sum a_i L_i - L_3 - L_4 - (L_3-mu)^2 h - (L_4-mu)^2 h - (x_1+x_2-r)^2 ht)
    // with L_i = ln x_i (the 1/(x_3 x_4) of the lognormals folded into the
    // exponent, c2 = a_3 + 1 and c3 = a_4 + 1).  The add of axis j is unrolled
    // with j known, so each axis takes only its own terms.
    // In double precision the lognormal terms are expanded, h (L - mu)^2 =
    // h L^2 - 2 h mu L + h mu^2 (c11, c12: the linear coefficients; c13: the
    // two constants, added by the first FMA), each axis's quadratic taken
    // as L (h L + lin) by two FMAs, and c10 is part of the Jacobian's
    // constant: five FP64 instructions per sample fewer, on the pipe that
    // bounds these kernels; the Jacobian itself (an integer product) is
    // multiplied into the exponential's fixed-point result (end_scaled), one
    // FP64 multiply fewer.  Single precision keeps the factored form (its
    // rounding would not survive the expansion's cancellation).
    static constexpr bool kWide = sizeof(R) == 8;
    // a logarithm per axis: the FP64 sampling loop runs its axes as a loop
    // (one copy of the per-axis code) instead of unrolling them
    static constexpr bool kRolled = kWide;
    struct S { R e; R x12; };
    __device__ static void begin(S& s) { s.e = R(0); s.x12 = R(0); }
    __device__ static void add(S& s, int j, R x, const FamParams& f)
    {
        const R L = RealOps<R>::log_(x);
        if constexpr (kWide) {
            if (j == 0) s.e = fma(f.c[0], L, f.c[13]);
            else if (j == 2 || j == 3) s.e = fma(L, fma(f.c[7], L, f.c[9 + j]), s.e);  // L (h L + lin) + e
            else s.e = fma(f.c[j], L, s.e);
        } else {
            s.e = j == 0 ? RealOps<R>::par(f, 0) * L : s.e + RealOps<R>::par(f, j) * L;
            if (j == 2 || j == 3) {
                const R z = L - RealOps<R>::par(f, 6);
                s.e += z * z * RealOps<R>::par(f, 7);
            }
        }
        if (j == 0) s.x12 = x;
        if (j == 1) s.x12 += x;
    }
    __device__ static R end(const S& s, uint32_t, const FamParams& f)
    {
        const R z = s.x12 - RealOps<R>::par(f, 8);
        if constexpr (kWide) return RealOps<R>::expm_(s.e + z * z * f.c[9]);  // c10: in the Jacobian
        else return RealOps<R>::par(f, 10) * RealOps<R>::expm_(s.e + z * z * RealOps<R>::par(f, 9));
    }
    // f J in double precision, J = (jm / 2^63) 2^je the integer Jacobian
    __device__ static double end_scaled(const S& s, const FamParams& f, uint64_t jm, int je)
    {
        const double z = s.x12 - f.c[8];
        return fx::fx_exp_neg_scaled(s.e + z * z * f.c[9], jm, je);
    }
};

// Interpolation tables (TABLE family): the point is clamped into the knot
// range, u = (x - lo) s with s = (n - 1)/(hi - lo), cell i = floor(u) (at
// most n - 2), t = u - i, and the value is (1 - t) v_i + t v_{i+1}
// (bilinear: the same on both axes).  The interpolant is continuous at the
// knots, so a point on a knot gives the same value from either cell.
template <typename R> struct TabOps;
template <> struct TabOps<double> {
    // Cell and fraction with one FP64 operation: u = x s - lo s by one FMA;
    // the floor of u (0 <= u < 2^31) and the fraction t = u - floor(u) are
    // taken from the bits of u's encoding (t normalised into a double with
    // integer operations), and the clamps are integer tests on those bits, so
    // no FP64 subtraction, conversion or compare is issued (GB300 runs 2 FP64
    // instructions per clock per SM against 64 integer ones).
    __device__ static void cell(double x, double s, double los, int n, int* i, double* t)
    {
        const double u = fma(x, s, -los);
        int64_t b = __double_as_longlong(u);
        if (b < 0) b = 0;                         // below the range (or -0): u = 0
        const int e = (int)((uint64_t)b >> 52) - 1023;
        if (e < 0) {                              // u < 1: cell 0, t = u
            *i = 0;
            *t = __longlong_as_double(b);
            return;
        }
        const int sh = 52 - e;
        const uint64_t M = ((uint64_t)b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int k = e < 31 ? (int)(M >> sh) : n;  // u >= 2^31 > n - 1 (also inf, NaN)
        if (k > n - 2) {                          // floor(u) >= n - 1: at or above the last knot
            *i = n - 2;
            *t = 1.0;
            return;
        }
        *i = k;
        // t = F 2^-sh for the fraction bits F < 2^sh: exact, normalised here
        const uint64_t F = M & ((1ull << sh) - 1ull);
        const int q = 63 - __clzll((long long)F);  // leading bit of F (q < sh <= 52)
        const uint64_t tb = ((uint64_t)(q - sh + 1022) << 52) + (F << (52 - q));
        *t = F ? __longlong_as_double((long long)tb) : 0.0;
    }
    __device__ static double interp1(const TableDesc& T, double x)
    {
        int i;
        double t;
        cell(x, T.s0, T.los0, T.n0, &i, &t);
        const double v0 = __ldg(T.v + i), v1 = __ldg(T.v + i + 1);
        return fma(t, v1 - v0, v0);
    }
    __device__ static double interp2(const TableDesc& T, double x, double y)
    {
        int i, k;
        double t, s;
        cell(x, T.s0, T.los0, T.n0, &i, &t);
        cell(y, T.s1, T.los1, T.n1, &k, &s);
        const double* r0 = T.v + (size_t)i * T.n1 + k;
        const double* r1 = r0 + T.n1;
        const double v00 = __ldg(r0), v01 = __ldg(r0 + 1), v10 = __ldg(r1), v11 = __ldg(r1 + 1);
        const double a = fma(t, v10 - v00, v00), b = fma(t, v11 - v01, v01);
        return fma(s, b - a, a);
    }
};
template <> struct TabOps<float> {
    __device__ static void cell(float x, float lo, float hi, float s, int n, int* i, float* t)
    {
        const float u = (fminf(fmaxf(x, lo), hi) - lo) * s;
        const int k = min((int)u, n - 2);
        *i = k;
        *t = u - (float)k;
    }
    __device__ static float interp1(const TableDesc& T, float x)
    {
        int i;
        float t;
        cell(x, T.lo0f, T.hi0f, T.s0f, T.n0, &i, &t);
        return (1.0f - t) * __ldg(T.vf + i) + t * __ldg(T.vf + i + 1);
    }
    __device__ static float interp2(const TableDesc& T, float x, float y)
    {
        int i, k;
        float t, s;
        cell(x, T.lo0f, T.hi0f, T.s0f, T.n0, &i, &t);
        cell(y, T.lo1f, T.hi1f, T.s1f, T.n1, &k, &s);
        const float* r0 = T.vf + (size_t)i * T.n1 + k;
        const float* r1 = r0 + T.n1;
        return (1.0f - t) * (1.0f - s) * __ldg(r0) + t * (1.0f - s) * __ldg(r1) + (1.0f - t) * s * __ldg(r0 + 1) +
               t * s * __ldg(r1 + 1);
    }
};

template <typename R> struct Family<MCUBES_F_TABLE, R> {
    // the coordinates are kept (registers: every index below is a
    // compile-time constant) and the factors evaluated at the end
    struct S { R x[kDMax]; };
    __device__ static void begin(S& s)
    {
#pragma unroll
        for (int j = 0; j < kDMax; ++j) s.x[j] = R(0);
    }
    __device__ static void add(S& s, int j, R x, const FamParams&) { s.x[j] = x; }
    __device__ static R sel(const S& s, int a)
    {
        R v = s.x[0];
#pragma unroll
        for (int j = 1; j < kDMax; ++j)
            if (a == j) v = s.x[j];
        return v;
    }
    __device__ static R end(const S& s, uint32_t, const FamParams& f)
    {
        R prod = RealOps<R>::par(f, 0);
        for (int q = 0; q < f.nf; ++q) {
            const TableDesc& T = f.tabs[f.tid[q]];
            const R xa = sel(s, f.ta[q]);
            if (f.tb[q] < 0) prod *= TabOps<R>::interp1(T, xa);
            else prod *= TabOps<R>::interp2(T, xa, sel(s, f.tb[q]));
        }
        return prod;
    }
};

// ---------------------------------------------------------------------------
// Compensated single-precision accumulator (Knuth's TwoSum; the pair holds
// about 48 significant bits).  Used for the per-thread sums over cubes of the
// mixed-precision path, which must not issue FP64 work per sample.
// ---------------------------------------------------------------------------
struct DFloat {
    float hi, lo;
    __device__ void add(float v)
    {
        const float s = __fadd_rn(hi, v);
        const float bp = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(v, bp));
        hi = s;
        lo = __fadd_rn(lo, err);
    }
    __device__ double value() const { return (double)hi + (double)lo; }
};

}  // namespace mc
