// refine_dev.cuh -- device pieces of the per-iteration finalisation shared
// by the single-integral and the batched refinement launches: fixed-order
// block sums, a double-double block scan, Weighted-Estimates with
// Check-Convergence (Alg. 2), and Adjust-Bin-Bounds of one axis (Alg. 2,
// Lepage 1978).
#pragma once

#include <cmath>

#include "mc_device.cuh"

namespace mc {
namespace refine_detail {

constexpr int kWarps = kRefineThreads / 32;
constexpr int kPerThread = (kNbMax + kRefineThreads - 1) / kRefineThreads;

// Deterministic block sum (each thread's value added in a fixed tree).
static __device__ __forceinline__ double block_sum(double v, double* scratch)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double w = lane < kWarps ? scratch[lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) w += __shfl_down_sync(0xffffffffu, w, off);
        if (lane == 0) scratch[32] = w;
    }
    __syncthreads();
    const double out = scratch[32];
    __syncthreads();
    return out;
}

// Fixed-order sums of N values over the first kRedThreads threads of the
// block (the other threads pass nothing and only meet the barriers; every
// thread of the block must call).  GB300's FP64 pipe takes one warp
// instruction per 16 cycles per SM whatever the number of active lanes, so
// the small reductions of the finalisation run on four warps, not sixteen.
constexpr int kRedThreads = 128;

template <int N>
static __device__ __forceinline__ void red4w(double (&v)[N])
{
    constexpr int kRedWarps = kRedThreads / 32;
    __shared__ double red[N][kRedWarps];
    __shared__ double out[N];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < kRedWarps) {
#pragma unroll
        for (int q = 0; q < N; ++q) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
            if (lane == 0) red[q][warp] = v[q];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            double t = red[q][0];
#pragma unroll
            for (int w = 1; w < kRedWarps; ++w) t += red[q][w];
            out[q] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < N; ++q) v[q] = out[q];
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Exact cumulative weights of the rebinning: each bin weight w in [0, 1] as an
// unsigned Q100 integer (128 bits; bits below 2^-100 dropped), their prefix
// sums exact (at most nb 2^100 < 2^110), so the order of the additions does
// not matter and the quantile tests are exact integer comparisons.
// ---------------------------------------------------------------------------
using u128 = unsigned __int128;

static __device__ __forceinline__ u128 q100_of(double w)  // 0 <= w < 2^27
{
    const uint64_t b = (uint64_t)__double_as_longlong(w);
    const int E = (int)(b >> 52);
    if (E == 0) return 0;                             // zero (or below 2^-1022)
    const uint64_t M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = E - 975;                           // w = (M << (E - 975)) 2^-100
    if (sh >= 0) return (u128)M << sh;                // sh < 75: below 2^128
    return sh > -53 ? (u128)(M >> -sh) : (u128)0;
}

// v rounded to the nearest double: one correctly rounded 64-bit conversion of
// the top word (a sticky bit stands for the rest) and an exact power-of-two
// scale.
static __device__ __forceinline__ double u128_to_double(u128 v)
{
    const uint64_t hi = (uint64_t)(v >> 64), lo = (uint64_t)v;
    if (hi == 0) return (double)lo;
    const int lz = __clzll((long long)hi);
    const u128 n = v << lz;
    const uint64_t top = (uint64_t)(n >> 64) | ((uint64_t)n != 0 ? 1ull : 0ull);
    const double scale = __longlong_as_double((long long)((uint64_t)(1023 + 64 - lz) << 52));  // 2^(64 - lz)
    return (double)top * scale;
}

static __device__ __forceinline__ u128 shfl_up_u128(u128 v, int off)
{
    const unsigned long long lo = __shfl_up_sync(0xffffffffu, (unsigned long long)v, off);
    const unsigned long long hi = __shfl_up_sync(0xffffffffu, (unsigned long long)(v >> 64), off);
    return ((u128)hi << 64) | (u128)lo;
}

// Inclusive prefix sum of the values w[0..n) (Q100) into c[0..n); thread t
// holds w[t kPerThread + i] in v[i] (zero beyond n).  The thread totals are
// scanned by warp shuffles and then across warps.  Exact, so any order gives
// the same sums.
static __device__ void u128_inclusive_scan(const u128 (&v)[kPerThread], u128* c, int n, u128* wtot)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int begin = t * kPerThread;
    u128 local = 0;
#pragma unroll
    for (int i = 0; i < kPerThread; ++i) local += v[i];
    u128 incl = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const u128 o = shfl_up_u128(incl, off);
        if (lane >= off) incl += o;
    }
    __syncthreads();
    if (lane == 31) wtot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        u128 x = lane < kWarps ? wtot[lane] : (u128)0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const u128 o = shfl_up_u128(x, off);
            if (lane >= off) x += o;
        }
        if (lane < kWarps) wtot[lane] = x;  // inclusive warp totals
    }
    __syncthreads();
    u128 run = incl - local + (warp > 0 ? wtot[warp - 1] : (u128)0);
#pragma unroll
    for (int i = 0; i < kPerThread; ++i) {
        const int k = begin + i;
        run += v[i];
        if (k < n) c[k] = run;
    }
    __syncthreads();
}

// Weighted-Estimates (inverse-variance weights, chi^2 per degree of freedom)
// and Check-Convergence over n recorded iterations: thread t < kRedThreads
// takes iterations t, t + kRedThreads, ..., keeps their weights (the
// reciprocals of the variances, formed in parallel: on GB300 a dependent
// FP64 division costs thousands of cycles) and the sums are fixed-order.
// Every thread of the block calls and gets the same values.
static __device__ bool weigh_and_check(const double* hI, const double* hV, int n, double rel_tol, double abs_tol,
                                       double* est, double* sigma, double* chi2_dof)
{
    double s4[4] = {0.0, 0.0, 0.0, 0.0};
    double w0 = 0.0, I0 = 0.0;  // this thread's first iteration, kept for the chi^2 pass
    const double inv_dof = n > 1 ? 1.0 / (double)(n - 1) : 0.0;  // off the dependent chain
    const int tmax = threadIdx.x < kRedThreads ? (n - (int)threadIdx.x + kRedThreads - 1) / kRedThreads : 0;
    for (int t = 0; t < tmax; ++t) {
        const int i = (int)threadIdx.x + t * kRedThreads;
        const double I = hI[i], V = hV[i];
        if (V == 0.0) {
            s4[0] += 1.0;
            s4[1] += I;
        } else {
            const double w = 1.0 / V;
            s4[2] += w;
            s4[3] += w * I;
            if (t == 0) w0 = w;
        }
        if (t == 0) I0 = I;
    }
    red4w<4>(s4);
    double I, sig, chi2 = 0.0;
    if (s4[0] > 0.0) {
        I = s4[1] / s4[0];
        sig = 0.0;
    } else {
        const double inv_sw = 1.0 / s4[2];
        I = s4[3] * inv_sw;
        sig = sqrt(inv_sw);
        if (n > 1) {
            double c[1] = {0.0};
            for (int t = 0; t < tmax; ++t) {
                const int i = (int)threadIdx.x + t * kRedThreads;
                const double z = (t == 0 ? I0 : hI[i]) - I;
                c[0] += z * z * (t == 0 ? w0 : 1.0 / hV[i]);
            }
            red4w<1>(c);
            chi2 = c[0] * inv_dof;
        }
    }
    *est = I;
    *sigma = sig;
    *chi2_dof = chi2;
    const double tol = fmax(abs_tol, rel_tol * fabs(I));
    return n >= 2 && sig <= tol;
}

// Where one integral's iteration results live (a single context's DevState,
// or one entry of a batch's state array plus its history arrays).
struct IterRecord {
    uint32_t* it;
    int* done;
    int* error;
    int* n;
    int* converged;
    double* estimate;
    double* sigma;
    double* chi2_dof;
    double* hist_I;
    double* hist_V;
    int cap;
    double rel_tol, abs_tol;
};

// Reduces nparts block partials (3 doubles each, fixed order) into the
// iteration estimate I = sum means / m and variance sum vars / m^2, records
// them, weighs all iterations, tests convergence and advances the iteration.
// With split > 1 the partials are (K, S1, S2) of cube slices, split
// consecutive ones per cube (sums of F - K over a slice of q = ceil(p/split)
// samples, the last slice shorter): each cube's slices are re-based on the
// first slice's shift and summed in order, then the cube's mean and the
// variance of that mean follow (UpdateVariance of Alg. 3).
static __device__ void finalize_iteration(const double* part, int nparts, double m, const IterRecord& r,
                                          int split = 1, double p = 0.0)
{
    double s01[2] = {0.0, 0.0};
    if (split > 1) {
        // thread t < kRedThreads merges cubes t, t + kRedThreads, ...: each
        // slice re-based on the cube's first shift and added in slice order,
        // eight slices' partials loaded ahead at a time; then the cube's mean
        // and the variance of that mean (UpdateVariance of Alg. 3) with the
        // reciprocals formed once (a dependent FP64 division costs thousands
        // of cycles on GB300)
        const int ncubes = nparts / split;
        const double q = ceil(p / split);
        const double inv_p = 1.0 / p, inv_var_den = inv_p / (p - 1.0);
        for (int cb = threadIdx.x; threadIdx.x < kRedThreads && cb < ncubes; cb += kRedThreads) {
            const double* v = part + 3 * (size_t)cb * split;
            const double K0 = v[0];
            double S1 = 0.0, S2 = 0.0;
            for (int k0 = 0; k0 < split; k0 += 8) {
                double a0[8], a1[8], a2[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int k = min(k0 + u, split - 1);
                    a0[u] = v[3 * k];
                    a1[u] = v[3 * k + 1];
                    a2[u] = v[3 * k + 2];
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int k = k0 + u;
                    if (k < split) {
                        const double n = fmin(q, fmax(p - q * k, 0.0));
                        const double dK = a0[u] - K0;
                        S2 += fma(dK, fma(n, dK, 2.0 * a1[u]), a2[u]);
                        S1 += fma(n, dK, a1[u]);
                    }
                }
            }
            s01[0] += K0 + S1 * inv_p;
            s01[1] += (S2 - S1 * S1 * inv_p) * inv_var_den;
        }
    } else {
        for (int b = threadIdx.x; threadIdx.x < kRedThreads && b < nparts; b += kRedThreads) {
            s01[0] += part[3 * (size_t)b + 0];
            s01[1] += part[3 * (size_t)b + 1];
        }
    }
    red4w<2>(s01);
    const double s0 = s01[0], s1 = s01[1];
    __shared__ int finite;
    if (threadIdx.x == 0) {
        const double I = s0 / m;
        const double V = s1 / (m * m);
        const int n = *r.n;
        if (n < r.cap) {
            r.hist_I[n] = I;
            r.hist_V[n] = V;
            *r.n = n + 1;
        }
        finite = isfinite(I) && isfinite(V);
        if (!finite) {
            *r.error = MCUBES_ENONFINITE;
            *r.done = 1;
        }
    }
    __syncthreads();  // the record and the flag are visible to the block
    if (finite) {
        double est, sig, chi2;
        const bool conv = weigh_and_check(r.hist_I, r.hist_V, *r.n, r.rel_tol, r.abs_tol, &est, &sig, &chi2);
        if (threadIdx.x == 0) {
            *r.estimate = est;
            *r.sigma = sig;
            *r.chi2_dof = chi2;
            if (conv) {
                *r.converged = 1;
                *r.done = 1;
            }
        }
    }
    if (threadIdx.x == 0) *r.it += 1;
}

// Three times the smoothed value of bin k: C_{k-1} + C_k + C_{k+1}; the ends
// 1.5 (C_0 + C_1) and 1.5 (C_{nb-2} + C_{nb-1}) (nb >= 2).
static __device__ __forceinline__ double smoothed3(const double* sC, int k, int nb)
{
    if (k == 0) return 1.5 * (sC[0] + sC[1]);
    if (k == nb - 1) return 1.5 * (sC[nb - 2] + sC[nb - 1]);
    return sC[k - 1] + sC[k] + sC[k + 1];
}

// Compressed weight ((r - 1)/ln r)^alpha of a bin, r = sm3 / total, as Q100
// (the library's log/exp: their FP64 work is a few instructions; CUDA's log
// and pow cost ~100 on a pipe that issues 2 per clock per SM).
static __device__ __forceinline__ u128 compressed_weight(double sm3, double inv_total, double alpha)
{
    const double r = sm3 * inv_total;
    double w;
    if (r <= 0.0) w = 0.0;
    else if (r >= 1.0) w = 1.0;
    else {
        const double q = (r - 1.0) / fx::fx_log(r);
        w = alpha == 1.5 ? q * sqrt(q) : fx::fx_exp(alpha * fx::fx_log(q));
    }
    return q100_of(w);
}

// New right edge of bin i - 1 (1 <= i < nb): the first bin k whose
// cumulative weight reaches i/nb of the total W (nb C_k >= i W), at the
// fraction (i W - nb C_{k-1}) / (nb w_k) of its width, in double-double.
static __device__ __forceinline__ DD rebin_edge(int i, int nb, u128 W, const u128* sCum, const double* sB,
                                                const double* sBlo)
{
    const u128 T = (u128)(uint64_t)i * W;
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((u128)(uint64_t)nb * sCum[mid] >= T) hi = mid; else lo = mid + 1;
    }
    const int k = lo;
    const u128 before = k > 0 ? (u128)(uint64_t)nb * sCum[k - 1] : (u128)0;  // < T
    const u128 wk = sCum[k] - (k > 0 ? sCum[k - 1] : (u128)0);
    const double frac = u128_to_double(T - before) / u128_to_double((u128)(uint64_t)nb * wk);
    const DD left = k > 0 ? DD{sB[k - 1], sBlo[k - 1]} : DD{0.0, 0.0};
    const DD width = dd_add(DD{sB[k], sBlo[k]}, DD{-left.hi, -left.lo});
    return dd_add(left, dd_scale(width, frac));
}

// Adjust-Bin-Bounds of one axis (Lepage 1978, as the paper's Alg. 2 cites):
// smooth the bin sums with their neighbours, normalise, compress with
// ((r - 1) / ln r)^alpha, then place the new right edges where the
// cumulative compressed weight reaches i / nb of its total, the weight of an
// old bin being spread evenly over it.  The smoothing keeps three times the
// neighbour mean (the normalisation removes the factor, and no division is
// issued per bin); the cumulative weight is exact in Q100 integers, so the
// bin of target i is the first k with nb C_k >= i W (W the total) and the
// fraction within it is (i W - nb C_{k-1}) / (nb w_k), both exact integers
// rounded once to doubles; the edge left + width * fraction is formed in
// double-double, so the new bin widths keep full double precision.  GB300
// issues 2 FP64 instructions per clock per SM and one block runs an axis:
// the integer form keeps the scan and the search off the FP64 pipe.
// The axis's histogram is the sum of nparts partials, element k of partial t
// at parts[t * stride + k] (float or double).  grid/grid_lo are this axis's
// edges (updated in place), hist_out receives the summed histogram.  The new
// edges are also written to the ncopy - 1 rows that follow (nb apart): the
// axes that share this axis's boundaries in m-Cubes1D (Sec. 3).
static __device__ void rebin_axis(const void* parts, size_t stride, int nparts, bool is_float, int nb, double alpha,
                           double* grid, double* grid_lo, double* hist_out, int* error, int* done, double* scratch,
                           int ncopy = 1)
{
    __shared__ double sC[kNbMax];
    __shared__ double sB[kNbMax];
    __shared__ double sBlo[kNbMax];
    __shared__ u128 sCum[kNbMax];   // inclusive cumulative compressed weights, Q100
    __shared__ u128 wtot[kWarps];
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        double acc = 0.0;
        if (is_float) {
            const float* ph = static_cast<const float*>(parts) + k;
            for (int b = 0; b < nparts; ++b) acc += (double)ph[b * stride];
        } else {
            const double* ph = static_cast<const double*>(parts) + k;
            for (int b = 0; b < nparts; ++b) acc += ph[b * stride];
        }
        sC[k] = acc;
        hist_out[k] = acc;
        sB[k] = grid[k];
        sBlo[k] = grid_lo[k];
    }
    __syncthreads();
    // three times the smoothed value: C_{k-1} + C_k + C_{k+1}; the ends 1.5 (C_0 + C_1)
    double sm3[kPerThread];
    double part = 0.0;
    for (int i = 0; i < kPerThread; ++i) {
        const int k = threadIdx.x * kPerThread + i;
        sm3[i] = k < nb ? smoothed3(sC, k, nb) : 0.0;
        part += sm3[i];  // fixed order: contiguous chunks per thread, then the tree
    }
    const double total = block_sum(part, scratch);
    if (!isfinite(total)) {
        if (threadIdx.x == 0) {
            *error = MCUBES_ENONFINITE;
            *done = 1;
        }
        return;
    }
    if (total <= 0.0) return;  // no information on this axis: grid unchanged
    const double inv_total = 1.0 / total;
    u128 wq[kPerThread];
#pragma unroll
    for (int i = 0; i < kPerThread; ++i) {
        const int k = threadIdx.x * kPerThread + i;
        wq[i] = k < nb ? compressed_weight(sm3[i], inv_total, alpha) : (u128)0;
    }
    u128_inclusive_scan(wq, sCum, nb, wtot);
    const u128 W = sCum[nb - 1];
    if (W == 0) {
        if (threadIdx.x == 0) {
            *error = MCUBES_ENONFINITE;
            *done = 1;
        }
        return;
    }
    double* out = grid;
    double* out_lo = grid_lo;
    for (int i = 1 + threadIdx.x; i < nb; i += blockDim.x) {
        const DD e = rebin_edge(i, nb, W, sCum, sB, sBlo);
        for (int r = 0; r < ncopy; ++r) {
            out[(size_t)r * nb + i - 1] = e.hi;
            out_lo[(size_t)r * nb + i - 1] = e.lo;
        }
    }
    if (threadIdx.x == 0) {
        for (int r = 0; r < ncopy; ++r) {
            out[(size_t)r * nb + nb - 1] = 1.0;
            out_lo[(size_t)r * nb + nb - 1] = 0.0;
        }
    }
}


}  // namespace refine_detail
}  // namespace mc
