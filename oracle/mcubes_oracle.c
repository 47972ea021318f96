/*
 * mcubes_oracle.c -- plain, slow, double-precision CPU oracle of the m-Cubes
 * VEGAS iteration (Sakiotis et al., "m-Cubes: An efficient and portable
 * implementation of multi-dimensional integration for GPUs", arXiv 2202.01753).
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists so that the CUDA path can be
 * checked against an independent statement of what the method computes.
 * Only the test suite, the package smoke check and the benchmark's CPU
 * baseline leg may load it.  It shares no code, header, table or constant
 * generator with the CUDA library; the two are written separately.
 *
 * Every function below cites the passage of the paper it follows.  Where the
 * paper is silent, the reading taken is stated next to the code:
 *   - the random numbers are Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3", SC'11), keyed by the
 *     64-bit seed, with counter (sample, cube, iteration, dimension block);
 *   - the map from the unit cube to the integration region is the piecewise
 *     linear VEGAS map of Lepage (1978), the reference the paper gives for
 *     its step from y to x (Alg. 1, Sec. 3);
 *   - the per-cube variance ("UpdateVariance", Alg. 3) is the unbiased
 *     variance of the cube's sample mean;
 *   - the grid refinement ("Adjust-Bin-Bounds", Alg. 2) is Lepage's
 *     smoothing, compression with exponent alpha, and equal-share rebinning;
 *   - iterations are combined with inverse-variance weights ("Weighted-
 *     Estimates", Alg. 2) and chi^2 per degree of freedom;
 *   - the m-Cubes1D variant (Sec. 3) keeps the histogram of axis 0 only,
 *     rebins that axis, and gives its boundaries to every axis.
 *
 * Compile with -ffp-contract=off: the only floating-point decisions that feed
 * an integer (none: the bin index is computed in exact integer arithmetic)
 * would otherwise depend on the compiler's fusing of multiply and add.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2
#define OR_ENONFINITE 4
#define OR_ENOCONV 5

#define OR_DMAX 12
#define OR_NBMAX 1024

/* integrand families (ids shared by value with the CUDA library's registry) */
#define OR_F_CONST 0
#define OR_F_GAUSS 1
#define OR_F_CORNER 2
#define OR_F_OSC 3
#define OR_F_PRODPEAK 4
#define OR_F_C0 5
#define OR_F_DISCONT 6
#define OR_F_COSMO6 7
#define OR_F_TABLE 8

/* ------------------------------------------------------------------------ */
/* Interpolation tables of the TABLE family (the paper's stateful           */
/* integrands, Sec. 6.1: integrands that read tabulated data at run time).  */
/* A table holds values at uniformly spaced knots: n0 knots over            */
/* [lo0, hi0] (and n1 over [lo1, hi1] for a 2-D table, values row-major,    */
/* v[i0 * n1 + i1]).  Its value at a point is the linear (bilinear)         */
/* interpolant of the knot values, the point first clamped into the table's */
/* range.  The oracle keeps pointers to the caller's arrays.                */
/* ------------------------------------------------------------------------ */
#define OR_TABLES_MAX 16
typedef struct {
    int ndim, n0, n1;
    double lo0, hi0, lo1, hi1;
    const double *v;
} or_table;
static or_table g_tables[OR_TABLES_MAX];
static int g_ntables = 0;

int oracle_set_tables(int n, const int *ndim, const int *n0, const int *n1, const double *lo0,
                      const double *hi0, const double *lo1, const double *hi1, const double *const *values)
{
    if (n < 0 || n > OR_TABLES_MAX) return OR_EINVAL;
    for (int t = 0; t < n; ++t) {
        if ((ndim[t] != 1 && ndim[t] != 2) || n0[t] < 2 || (ndim[t] == 2 && n1[t] < 2)) return OR_EINVAL;
        if (!(lo0[t] < hi0[t]) || (ndim[t] == 2 && !(lo1[t] < hi1[t])) || !values[t]) return OR_EINVAL;
    }
    for (int t = 0; t < n; ++t) {
        or_table tb = {ndim[t], n0[t], ndim[t] == 2 ? n1[t] : 1, lo0[t], hi0[t], lo1[t], hi1[t], values[t]};
        g_tables[t] = tb;
    }
    g_ntables = n;
    return OR_OK;
}

/* cell index and fraction of x on n knots over [lo, hi]: x clamped, then   */
/* u = (x - lo) / h with h = (hi - lo)/(n - 1), i = floor(u) (at most n-2), */
/* t = u - i.  (The interpolant is continuous at the knots, so which of two */
/* cells a point on a knot is given to does not change the value.)          */
static void table_cell(double x, int n, double lo, double hi, int *i, double *t)
{
    if (x < lo) x = lo;
    if (x > hi) x = hi;
    double h = (hi - lo) / (double)(n - 1);
    double u = (x - lo) / h;
    int k = (int)floor(u);
    if (k > n - 2) k = n - 2;
    if (k < 0) k = 0;
    *i = k;
    *t = u - (double)k;
}

static double table_value(const or_table *tb, double xa, double xb)
{
    int i, k;
    double t, s;
    table_cell(xa, tb->n0, tb->lo0, tb->hi0, &i, &t);
    if (tb->ndim == 1) return (1.0 - t) * tb->v[i] + t * tb->v[i + 1];
    table_cell(xb, tb->n1, tb->lo1, tb->hi1, &k, &s);
    const double *r0 = tb->v + (size_t)i * tb->n1, *r1 = r0 + tb->n1;
    return (1.0 - t) * (1.0 - s) * r0[k] + t * (1.0 - s) * r1[k] + (1.0 - t) * s * r0[k + 1] + t * s * r1[k + 1];
}

/* ------------------------------------------------------------------------ */
/* Double-double numbers (an unevaluated sum hi + lo; Dekker 1971, Knuth     */
/* TAOCP vol. 2 Sec. 4.2.2).  Grid edges are kept in this form so that a    */
/* narrow bin's width, the difference of two edges near the same value,    */
/* keeps full relative precision (the Jacobian is a product of widths);    */
/* the cumulative bin weights of the rebinning are kept in it so that the   */
/* quantile edges are exact to about 2^-104 of the total weight, whatever   */
/* the order of addition.                                                   */
/* ------------------------------------------------------------------------ */
typedef struct { double hi, lo; } ddnum;
static ddnum dd_two_sum(double a, double b)
{
    double s = a + b, bb = s - a;
    ddnum r = {s, (a - (s - bb)) + (b - bb)};
    return r;
}
static ddnum dd_norm(double hi, double lo)
{
    double s = hi + lo;
    ddnum r = {s, lo - (s - hi)};
    return r;
}
static ddnum dd_add(ddnum a, ddnum b)
{
    ddnum s = dd_two_sum(a.hi, b.hi);
    return dd_norm(s.hi, s.lo + a.lo + b.lo);
}
static ddnum dd_neg(ddnum a) { ddnum r = {-a.hi, -a.lo}; return r; }
static ddnum dd_mul_d(ddnum a, double b)
{
    double p = a.hi * b;
    double e = fma(a.hi, b, -p);
    return dd_norm(p, e + a.lo * b);
}
static ddnum dd_div_d(ddnum a, double b)
{
    double q1 = a.hi / b;
    ddnum r = dd_add(a, dd_neg(dd_mul_d((ddnum){q1, 0.0}, b)));
    double q2 = (r.hi + r.lo) / b;
    return dd_norm(q1, q2);
}
static int dd_ge(ddnum a, ddnum b) { return a.hi > b.hi || (a.hi == b.hi && a.lo >= b.lo); }

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. 3.3 and Table 2).               */
/* Alg. 3 seeds a generator per thread but names none;                      */
/* this counter-based one makes every sample reproducible from    */
/* (seed, iteration, cube, sample) alone.                                    */
/* ------------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                          uint32_t out[4])
{
    const uint32_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u; /* SC'11 multipliers */
    const uint32_t bump0 = 0x9E3779B9u, bump1 = 0xBB67AE85u; /* golden ratio, sqrt(3)-1 */
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += bump0; k1 += bump1; }
        uint64_t prod0 = (uint64_t)mult0 * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)mult1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* The d random words of sample s of cube c in iteration it: word j is word
 * (j mod 4) of the Philox block with counter (s, c, it, j div 4). */
void oracle_sample_words(uint64_t seed, uint32_t it, uint32_t cube, uint32_t s,
                         int d, uint32_t *words)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int b = 0; 4 * b < d; ++b) {
        uint32_t ctr[4] = {s, cube, it, (uint32_t)b};
        uint32_t out[4];
        oracle_philox4x32_10(ctr, key, out);
        for (int q = 0; q < 4 && 4 * b + q < d; ++q) words[4 * b + q] = out[q];
    }
}

/* ------------------------------------------------------------------------ */
/* Geometry (Alg. 2: g = (maxcalls/2)^(1/d), m = g^d, p = maxcalls/m).       */
/* Reading: g is the largest integer with g^d <= ncall/2 (at least 1), cut   */
/* down so that m fits a 32-bit cube counter and nb*g <= 2^31; p is          */
/* floor(ncall/m) but at least 2, because a cube's variance needs 2 samples. */
/* ------------------------------------------------------------------------ */
static int ipow_le(int64_t g, int d, uint64_t limit, uint64_t *out)
{
    /* out = g^d if g^d <= limit; returns 0 on overflow past limit */
    uint64_t v = 1;
    for (int i = 0; i < d; ++i) {
        if ((uint64_t)g != 0 && v > limit / (uint64_t)g) return 0;
        v *= (uint64_t)g;
        if (v > limit) return 0;
    }
    *out = v;
    return 1;
}

int oracle_geometry(int d, int64_t ncall, int64_t g_override, int nb,
                    int64_t *g_out, int64_t *m_out, int64_t *p_out)
{
    if (d < 1 || d > OR_DMAX || ncall < 2 || nb < 2 || nb > OR_NBMAX) return OR_EINVAL;
    const uint64_t m_limit = 0xFFFFFFFFull;              /* cube index is a 32-bit counter */
    const int64_t g_limit = ((int64_t)1 << 31) / nb;      /* nb*g <= 2^31 */
    int64_t g;
    uint64_t m = 0;
    if (g_override > 0) {
        g = g_override;
        if (g > g_limit || !ipow_le(g, d, m_limit, &m)) return OR_EINVAL;
    } else {
        /* largest g in [1, g_limit] with g^d <= min(ncall/2, 2^32-1): bisection */
        uint64_t half = (uint64_t)ncall / 2;
        uint64_t cap = half < m_limit ? half : m_limit;
        uint64_t tmp;
        int64_t lo = 1, hi = g_limit;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo + 1) / 2;
            if (ipow_le(mid, d, cap, &tmp)) lo = mid; else hi = mid - 1;
        }
        g = lo;
        ipow_le(g, d, m_limit, &m);
    }
    int64_t p = ncall / (int64_t)m;
    if (p < 2) p = 2;
    if (p > 0xFFFFFFFFll) return OR_EINVAL; /* sample index is a 32-bit counter */
    *g_out = g;
    *m_out = (int64_t)m;
    *p_out = p;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Init-Bins (Alg. 2; Sec. 4): every axis starts as nb bins of equal width, */
/* kept as their right edges.  B is [d][nb], in unit coordinates.           */
/* ------------------------------------------------------------------------ */
void oracle_init_grid(int d, int nb, double *B, double *Blo)
{
    /* right edge (k+1)/nb as hi + lo: hi rounded, lo the rounded remainder */
    for (int j = 0; j < d; ++j) {
        for (int k = 0; k < nb; ++k) {
            double hi = (double)(k + 1) / (double)nb;
            double rem = fma(-hi, (double)nb, (double)(k + 1)); /* exact */
            if (k == nb - 1) { hi = 1.0; rem = 0.0; }
            B[j * nb + k] = hi;
            if (Blo) Blo[j * nb + k] = rem / (double)nb;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Position of one coordinate (Alg. 1, the step taking y to x; Alg. 3,      */
/* Get-Bin-ID).  Reading: the point lies in sub-cube digit c of this axis  */
/* (g equal intervals that never move, Sec. 4) at offset u = (w + 1/2)/2^32  */
/* inside it, so y = (c + u)/g.  Its bin is k = floor(nb*y), computed with   */
/* exact integers, and phi = nb*y - k is its position inside the bin.        */
/* ------------------------------------------------------------------------ */
void oracle_bin_of(uint32_t c, uint32_t w, int64_t g, int nb, int *k_out, double *phi_out)
{
    typedef unsigned __int128 u128;
    /* nb*y = nb*(c*2^33 + 2w + 1) / (g*2^33) exactly */
    u128 num = (u128)(uint64_t)nb * (((u128)c << 33) + 2 * (u128)w + 1);
    u128 den = (u128)(uint64_t)g << 33;
    *k_out = (int)(num / den);
    *phi_out = (double)(num % den) / (double)den;
}

/* Lepage's map through the bin grid of one axis: bin k spans
 * [B[k-1], B[k]] (B[-1] = 0); x = lo + (hi-lo)*(left + width*phi) and the
 * axis contributes (hi-lo)*nb*width to the Jacobian.  The edges are
 * double-double (Blo may be NULL: zero low parts). */
static void map_axis(const double *Bj, const double *Blj, int nb, double lo, double hi, int k,
                     double phi, double *x, double *jac)
{
    ddnum left = {0.0, 0.0}, right = {Bj[k], Blj ? Blj[k] : 0.0};
    if (k > 0) { left.hi = Bj[k - 1]; left.lo = Blj ? Blj[k - 1] : 0.0; }
    ddnum wd = dd_add(right, dd_neg(left));
    double width = wd.hi + wd.lo;
    *x = lo + (hi - lo) * (left.hi + width * phi);
    *jac = (hi - lo) * (double)nb * width;
}

/* ------------------------------------------------------------------------ */
/* Integrands.  The test families of Sec. 5 (eqs. 1-6, Genz's oscillatory,  */
/* product peak, corner peak, Gaussian, C0 and discontinuous families, and   */
/* f_A, f_B of Table 1) in parameterised form, plus a six-dimensional        */
/* power-law x lognormal x ridge integrand standing in for the cosmology     */
/* integrand of Sec. 6.1 and a constant.  Parameter layouts:                 */
/*   CONST    [v]                      f = v                                 */
/*   GAUSS    [A, mu_1..d, sig_1..d]   f = A prod exp(-(x-mu)^2/(2 sig^2))   */
/*   CORNER   [a_1..d]                 f = (1 + sum a x)^(-(d+1))            */
/*   OSC      [u, a_1..d]              f = cos(2 pi u + sum a x)             */
/*   PRODPEAK [c_1..d, w_1..d]         f = prod 1/(c^-2 + (x-w)^2)           */
/*   C0       [c_1..d, w_1..d]         f = exp(-sum c |x-w|)                 */
/*   DISCONT  [c_1..d, w_1..d]         f = exp(sum c x) if all x < w, else 0 */
/*   COSMO6   [a_1..6, mu, s, r, t]    f = prod x^-a * LN(x3) LN(x4)         */
/*                                         * exp(-(x1+x2-r)^2/(2 t^2)),      */
/*            LN(z) = exp(-(ln z - mu)^2/(2 s^2)) / (z s sqrt(2 pi))         */
/*   TABLE    [c, nf, (tab, a, b) x nf] f = c prod_q T_tab_q(x_a_q [, x_b_q]) */
/*            (axes 0-based; b = -1 for a 1-D table; 1 <= nf <= 10)          */
/* ------------------------------------------------------------------------ */
int oracle_nparams(int id, int d)
{
    switch (id) {
    case OR_F_CONST: return 1;
    case OR_F_GAUSS: return 1 + 2 * d;
    case OR_F_CORNER: return d;
    case OR_F_OSC: return 1 + d;
    case OR_F_PRODPEAK: case OR_F_C0: case OR_F_DISCONT: return 2 * d;
    case OR_F_COSMO6: return d == 6 ? 10 : -1;
    case OR_F_TABLE: return 0;  /* variable: 2 + 3 nf, checked by oracle_table_params */
    default: return -1;
    }
}

/* The TABLE family's params (count np) against the tables set: returns 1   */
/* if every factor names a table of the right dimension and valid axes.    */
int oracle_table_params(const double *par, int np, int d)
{
    if (np < 2) return 0;
    int nf = (int)par[1];
    if ((double)nf != par[1] || nf < 1 || nf > 10 || np != 2 + 3 * nf) return 0;
    for (int q = 0; q < nf; ++q) {
        double tq = par[2 + 3 * q], aq = par[3 + 3 * q], bq = par[4 + 3 * q];
        int t = (int)tq, a = (int)aq, b = (int)bq;
        if ((double)t != tq || (double)a != aq || (double)b != bq) return 0;
        if (t < 0 || t >= g_ntables || a < 0 || a >= d) return 0;
        if (g_tables[t].ndim == 1 && b != -1) return 0;
        if (g_tables[t].ndim == 2 && (b < 0 || b >= d || b == a)) return 0;
    }
    return 1;
}

double oracle_integrand(int id, const double *par, int d, const double *x)
{
    const double pi = 3.14159265358979323846;
    switch (id) {
    case OR_F_CONST:
        return par[0];
    case OR_F_GAUSS: {
        double f = par[0];
        for (int i = 0; i < d; ++i) {
            double z = x[i] - par[1 + i], s = par[1 + d + i];
            f *= exp(-(z * z) / (2.0 * s * s));
        }
        return f;
    }
    case OR_F_CORNER: {
        double t = 1.0;
        for (int i = 0; i < d; ++i) t += par[i] * x[i];
        return pow(t, -(double)(d + 1));
    }
    case OR_F_OSC: {
        double t = 2.0 * pi * par[0];
        for (int i = 0; i < d; ++i) t += par[1 + i] * x[i];
        return cos(t);
    }
    case OR_F_PRODPEAK: {
        double f = 1.0;
        for (int i = 0; i < d; ++i) {
            double c = par[i], z = x[i] - par[d + i];
            f *= 1.0 / (1.0 / (c * c) + z * z);
        }
        return f;
    }
    case OR_F_C0: {
        double t = 0.0;
        for (int i = 0; i < d; ++i) t += par[i] * fabs(x[i] - par[d + i]);
        return exp(-t);
    }
    case OR_F_DISCONT: {
        double t = 0.0;
        for (int i = 0; i < d; ++i) {
            if (!(x[i] < par[d + i])) return 0.0;
            t += par[i] * x[i];
        }
        return exp(t);
    }
    case OR_F_COSMO6: {
        double f = 1.0;
        for (int i = 0; i < 6; ++i) f *= pow(x[i], -par[i]);
        double mu = par[6], s = par[7], r = par[8], t = par[9];
        for (int i = 2; i < 4; ++i) {
            double l = log(x[i]) - mu;
            f *= exp(-(l * l) / (2.0 * s * s)) / (x[i] * s * sqrt(2.0 * pi));
        }
        double z = x[0] + x[1] - r;
        f *= exp(-(z * z) / (2.0 * t * t));
        return f;
    }
    case OR_F_TABLE: {
        double f = par[0];
        int nf = (int)par[1];
        for (int q = 0; q < nf; ++q) {
            const or_table *tb = &g_tables[(int)par[2 + 3 * q]];
            int a = (int)par[3 + 3 * q], b = (int)par[4 + 3 * q];
            f *= table_value(tb, x[a], b >= 0 ? x[b] : 0.0);
        }
        return f;
    }
    default:
        return NAN;
    }
}

/* ------------------------------------------------------------------------ */
/* Compensated (Neumaier) summation, so that the oracle's sums are exact to  */
/* about one rounding whatever the order the CUDA path adds in.              */
/* ------------------------------------------------------------------------ */
typedef struct { double s, c; } ksum;
static void ks_add(ksum *a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}
static double ks_val(const ksum *a) { return a->s + a->c; }

/* ------------------------------------------------------------------------ */
/* One V-Sample pass (Alg. 3, lines of the per-thread loop; Alg. 1 lines     */
/* 2-8) over cubes [cube_begin, cube_end) of one iteration.                  */
/*   sums_out[0] = sum over the cubes of the cube mean of F = f(x) J          */
/*   sums_out[1] = sum over the cubes of the variance of that mean           */
/*   sums_out[2] = sum over the cubes of |cube mean| (conditioning of [0])   */
/* Adjusting iterations (adjust != 0) also add F^2 of every sample to       */
/* C[j][k_j] for every axis j (Alg. 3: the bin contribution is the square   */
/* of the sample's estimate; the printed index C[b[j]] drops the axis and   */
/* is read as C[j][b[j]], one histogram per axis), and count hits H[j][k_j].*/
/* C and H are [d][nb], added to (not cleared); either may be NULL.  B/Blo */
/* are the grid's double-double right edges ([d][nb]; Blo may be NULL).     */
/* Returns OR_ENONFINITE if any F is not finite.                             */
/* ------------------------------------------------------------------------ */
/* one_dim != 0 selects the m-Cubes1D variant (Sec. 3, "The m-Cubes1D     */
/* variant"): every axis shares one set of bin boundaries, so only axis 0  */
/* keeps a histogram: C[0][k_0] (and H[0][k_0]) alone are added to; the    */
/* map itself is unchanged (the caller passes a grid whose rows are equal).*/
typedef struct {
    int id;
    const double *params;
    int d, nb;
    const double *lo, *hi;
    int64_t g, m, p;
    uint64_t seed;
    int one_dim;
} oracle_problem;

int oracle_vsample(const oracle_problem *pb, const double *B, const double *Blo, uint32_t it, int adjust,
                   uint64_t cube_begin, uint64_t cube_end, double *sums_out,
                   double *C, uint64_t *H)
{
    const int d = pb->d, nb = pb->nb;
    const int64_t p = pb->p;
    double *F = (double *)malloc(sizeof(double) * (size_t)p);
    ksum *Cs = NULL;
    if (!F) return OR_ENOMEM;
    if (adjust && C) {
        Cs = (ksum *)calloc((size_t)d * nb, sizeof(ksum));
        if (!Cs) { free(F); return OR_ENOMEM; }
        for (int i = 0; i < d * nb; ++i) Cs[i].s = C[i];
    }
    ksum Isum = {0, 0}, Vsum = {0, 0}, Asum = {0, 0};
    int status = OR_OK;
    uint32_t words[OR_DMAX];
    uint32_t digit[OR_DMAX];
    int kbin[OR_DMAX];
    double x[OR_DMAX];
    for (uint64_t c = cube_begin; c < cube_end; ++c) {
        /* sub-cube c has digits c_j in base g, axis 0 fastest */
        uint64_t rest = c;
        for (int j = 0; j < d; ++j) { digit[j] = (uint32_t)(rest % (uint64_t)pb->g); rest /= (uint64_t)pb->g; }
        for (int64_t s = 0; s < p; ++s) {
            oracle_sample_words(pb->seed, it, (uint32_t)c, (uint32_t)s, d, words);
            double jac = 1.0;
            for (int j = 0; j < d; ++j) {
                double phi, jj;
                oracle_bin_of(digit[j], words[j], pb->g, nb, &kbin[j], &phi);
                map_axis(B + (size_t)j * nb, Blo ? Blo + (size_t)j * nb : NULL, nb, pb->lo[j], pb->hi[j],
                         kbin[j], phi, &x[j], &jj);
                jac *= jj;
            }
            double v = oracle_integrand(pb->id, pb->params, d, x) * jac;
            if (!isfinite(v)) status = OR_ENONFINITE;
            F[s] = v;
            if (adjust) {
                const int hist_axes = pb->one_dim ? 1 : d;
                for (int j = 0; j < hist_axes; ++j) {
                    if (Cs) ks_add(&Cs[j * nb + kbin[j]], v * v);
                    if (H) H[j * nb + kbin[j]] += 1;
                }
            }
        }
        /* UpdateVariance (Alg. 3): cube mean and the unbiased variance of
         * that mean, by the two-pass definition */
        ksum m1 = {0, 0};
        for (int64_t s = 0; s < p; ++s) ks_add(&m1, F[s]);
        double mean = ks_val(&m1) / (double)p;
        ksum m2 = {0, 0};
        for (int64_t s = 0; s < p; ++s) { double z = F[s] - mean; ks_add(&m2, z * z); }
        double var = ks_val(&m2) / ((double)p * (double)(p - 1));
        ks_add(&Isum, mean);
        ks_add(&Vsum, var);
        ks_add(&Asum, fabs(mean));
    }
    if (Cs) {
        for (int i = 0; i < d * nb; ++i) C[i] = ks_val(&Cs[i]);
        free(Cs);
    }
    sums_out[0] = ks_val(&Isum);
    sums_out[1] = ks_val(&Vsum);
    sums_out[2] = ks_val(&Asum);
    free(F);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Adjust-Bin-Bounds (Alg. 2; Sec. 3: bins with large contributions are     */
/* made smaller), following Lepage (1978): smooth the per-bin sums with     */
/* their neighbours, normalise, compress with exponent alpha, then place    */
/* new right edges so that every new bin holds an equal share of the        */
/* compressed weight, the weight of an old bin being spread evenly over it. */
/* Edge i (1..nb-1) lies where the cumulative weight reaches i/nb of the    */
/* total: in the first bin k whose cumulative weight reaches that target,   */
/* at fraction (target - weight before k) / w_k of its width.               */
/* The edges Bj/Blj ([nb], double-double) are updated in place.  Returns 0 */
/* on success, 1 if the histogram of the axis was all zero (left            */
/* unchanged), OR_ENONFINITE if it was not finite (left unchanged).         */
/* ------------------------------------------------------------------------ */
int oracle_rebin_axis(int nb, double alpha, const double *Cj, double *Bj, double *Blj)
{
    double *sm = (double *)malloc(sizeof(double) * nb * 4);
    ddnum *cum = (ddnum *)malloc(sizeof(ddnum) * (nb + 1));
    if (!sm || !cum) { free(sm); free(cum); return OR_ENOMEM; }
    double *w = sm + nb, *newB = sm + 2 * nb, *newL = sm + 3 * nb;
    /* smoothing */
    if (nb == 1) sm[0] = Cj[0];
    else {
        sm[0] = (Cj[0] + Cj[1]) / 2.0;
        for (int k = 1; k < nb - 1; ++k) sm[k] = (Cj[k - 1] + Cj[k] + Cj[k + 1]) / 3.0;
        sm[nb - 1] = (Cj[nb - 2] + Cj[nb - 1]) / 2.0;
    }
    double total = 0.0;
    for (int k = 0; k < nb; ++k) total += sm[k];
    if (!isfinite(total)) { free(sm); free(cum); return OR_ENONFINITE; }
    if (total <= 0.0) { free(sm); free(cum); return 1; }
    /* normalisation and compression */
    for (int k = 0; k < nb; ++k) {
        double r = sm[k] / total;
        double v;
        if (r <= 0.0) v = 0.0;
        else if (r == 1.0) v = 1.0;
        else v = pow((r - 1.0) / log(r), alpha);
        w[k] = v;
    }
    /* cumulative weight: cum[k] = w_0 + ... + w_{k-1} */
    cum[0].hi = 0.0;
    cum[0].lo = 0.0;
    for (int k = 0; k < nb; ++k) cum[k + 1] = dd_add(cum[k], (ddnum){w[k], 0.0});
    ddnum wsum = cum[nb];
    if (!(wsum.hi > 0.0) || !isfinite(wsum.hi)) { free(sm); free(cum); return OR_ENONFINITE; }
    /* equal-share rebinning along the cumulative weight */
    int k = 0;
    for (int i = 1; i < nb; ++i) {
        ddnum target = dd_div_d(dd_mul_d(wsum, (double)i), (double)nb);
        while (k < nb - 1 && !dd_ge(cum[k + 1], target)) ++k;
        ddnum rem = dd_add(target, dd_neg(cum[k]));
        ddnum left = {0.0, 0.0}, right = {Bj[k], Blj[k]};
        if (k > 0) { left.hi = Bj[k - 1]; left.lo = Blj[k - 1]; }
        ddnum width = dd_add(right, dd_neg(left));
        double frac = (rem.hi + rem.lo) / w[k];
        if (frac > 1.0) frac = 1.0;
        if (frac < 0.0) frac = 0.0;
        ddnum e = dd_add(left, dd_mul_d(width, frac));
        newB[i - 1] = e.hi;
        newL[i - 1] = e.lo;
    }
    newB[nb - 1] = 1.0;
    newL[nb - 1] = 0.0;
    memcpy(Bj, newB, sizeof(double) * nb);
    memcpy(Blj, newL, sizeof(double) * nb);
    free(sm);
    free(cum);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Weighted-Estimates and Check-Convergence (Alg. 2; Sec. 5.1 uses the       */
/* normalised standard deviation as the stopping rule).  Reading: weights    */
/* 1/sigma_it^2; I = sum w I_it / sum w; sigma = (sum w)^(-1/2);             */
/* chi^2/dof = sum w (I_it - I)^2 / (n - 1) (0 when n = 1).  Iterations with */
/* zero variance are exact: if any exists, I is their mean and sigma = 0.    */
/* Converged when n >= 2 and sigma <= max(abs_tol, rel_tol |I|).             */
/* ------------------------------------------------------------------------ */
void oracle_weighted(int n, const double *I_it, const double *var_it, double rel_tol,
                     double abs_tol, double *est, double *sigma, double *chi2_dof,
                     int *converged)
{
    int n_exact = 0;
    double exact_sum = 0.0;
    for (int i = 0; i < n; ++i) if (var_it[i] == 0.0) { ++n_exact; exact_sum += I_it[i]; }
    double I, sig, chi2 = 0.0;
    if (n_exact > 0) {
        I = exact_sum / n_exact;
        sig = 0.0;
    } else {
        double sw = 0.0, swi = 0.0;
        for (int i = 0; i < n; ++i) { double w = 1.0 / var_it[i]; sw += w; swi += w * I_it[i]; }
        I = swi / sw;
        sig = sqrt(1.0 / sw);
        if (n > 1) {
            for (int i = 0; i < n; ++i) { double z = I_it[i] - I; chi2 += z * z / var_it[i]; }
            chi2 /= (double)(n - 1);
        }
    }
    *est = I;
    *sigma = sig;
    *chi2_dof = chi2;
    double tol = rel_tol * fabs(I);
    if (abs_tol > tol) tol = abs_tol;
    *converged = (n >= 2 && sig <= tol) ? 1 : 0;
}

/* ------------------------------------------------------------------------ */
/* The m-Cubes driver (Alg. 2): ita adjusting iterations, then plain ones,   */
/* itmax in all, stopping early once converged.  Reading of the loop bounds: */
/* iterations it = 0 .. itmax-1, adjusting while it < ita.                   */
/* Outputs (any pointer may be NULL): res = {estimate, sigma, chi2/dof},    */
/* iters_out = iterations run, conv_out = converged flag, trace_I/trace_var  */
/* (itmax entries) = per-iteration estimate and variance, B_out ([d][nb])   */
/* = final grid, C_out ([d][nb]) = histogram of the last adjusting          */
/* iteration.                                                                */
/* one_dim != 0 runs the m-Cubes1D variant (Sec. 3): the histogram of axis  */
/* 0 alone is kept, that axis is rebinned, and its new boundaries become    */
/* every axis's boundaries, so that all axes always share one grid.         */
/* ------------------------------------------------------------------------ */
int oracle_integrate(int id, const double *params, int d, const double *lo, const double *hi,
                     int64_t ncall, int itmax, int ita, int nb, int64_t g_override,
                     double alpha, uint64_t seed, double rel_tol, double abs_tol,
                     double *res, int *iters_out, int *conv_out, int64_t *geom_out,
                     double *trace_I, double *trace_var, double *B_out, double *C_out, int one_dim)
{
    if (itmax < 1 || d < 1 || d > OR_DMAX || nb < 2 || nb > OR_NBMAX) return OR_EINVAL;
    if (oracle_nparams(id, d) < 0) return OR_EINVAL;
    if (id == OR_F_TABLE) {
        if (!(params[1] >= 1.0 && params[1] <= 10.0)) return OR_EINVAL;
        if (!oracle_table_params(params, 2 + 3 * (int)params[1], d)) return OR_EINVAL;
    }
    for (int j = 0; j < d; ++j) if (!(lo[j] < hi[j]) || !isfinite(lo[j]) || !isfinite(hi[j])) return OR_EINVAL;
    int64_t g, m, p;
    int st = oracle_geometry(d, ncall, g_override, nb, &g, &m, &p);
    if (st) return st;
    if (geom_out) { geom_out[0] = g; geom_out[1] = m; geom_out[2] = p; }
    double *B = (double *)malloc(sizeof(double) * d * nb);
    double *Blo = (double *)malloc(sizeof(double) * d * nb);
    double *C = (double *)malloc(sizeof(double) * d * nb);
    double *hI = (double *)malloc(sizeof(double) * itmax);
    double *hV = (double *)malloc(sizeof(double) * itmax);
    if (!B || !Blo || !C || !hI || !hV) { free(B); free(Blo); free(C); free(hI); free(hV); return OR_ENOMEM; }
    oracle_init_grid(d, nb, B, Blo);
    oracle_problem pb = {id, params, d, nb, lo, hi, g, m, p, seed, one_dim};
    double est = 0, sig = 0, chi2 = 0;
    int conv = 0, n = 0;
    st = OR_OK;
    for (int it = 0; it < itmax; ++it) {
        int adjust = it < ita;
        double sums[3];
        if (adjust) memset(C, 0, sizeof(double) * d * nb);
        int s = oracle_vsample(&pb, B, Blo, (uint32_t)it, adjust, 0, (uint64_t)m, sums, adjust ? C : NULL, NULL);
        double I_it = sums[0] / (double)m;
        double V_it = sums[1] / ((double)m * (double)m);
        hI[n] = I_it;
        hV[n] = V_it;
        ++n;
        if (trace_I) trace_I[it] = I_it;
        if (trace_var) trace_var[it] = V_it;
        if (s == OR_ENONFINITE || !isfinite(I_it) || !isfinite(V_it)) { st = OR_ENONFINITE; break; }
        oracle_weighted(n, hI, hV, rel_tol, abs_tol, &est, &sig, &chi2, &conv);
        if (adjust) {
            if (C_out) memcpy(C_out, C, sizeof(double) * d * nb);
            const int rebinned = one_dim ? 1 : d;
            for (int j = 0; j < rebinned; ++j) {
                int r = oracle_rebin_axis(nb, alpha, C + (size_t)j * nb, B + (size_t)j * nb, Blo + (size_t)j * nb);
                if (r == OR_ENONFINITE) st = OR_ENONFINITE;
            }
            for (int j = rebinned; j < d; ++j) {   /* m-Cubes1D: the shared boundaries */
                memcpy(B + (size_t)j * nb, B, sizeof(double) * nb);
                memcpy(Blo + (size_t)j * nb, Blo, sizeof(double) * nb);
            }
            if (st) break;
        }
        if (conv) break;
    }
    if (res) { res[0] = est; res[1] = sig; res[2] = chi2; }
    if (iters_out) *iters_out = n;
    if (conv_out) *conv_out = conv;
    if (B_out) memcpy(B_out, B, sizeof(double) * d * nb);
    free(B); free(Blo); free(C); free(hI); free(hV);
    if (st) return st;
    return conv ? OR_OK : OR_ENOCONV;
}
