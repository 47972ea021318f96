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

static __device__ __forceinline__ DD dd_shfl_up(DD v, int off)
{
    return DD{__shfl_up_sync(0xffffffffu, v.hi, off), __shfl_up_sync(0xffffffffu, v.lo, off)};
}

// Inclusive double-double prefix sum of w[0..n) into (chi, clo), fixed
// order: each thread adds kPerThread consecutive values, the thread totals
// are scanned by warp shuffles and then across warps.
static __device__ void dd_inclusive_scan(const double* w, double* chi, double* clo, int n, DD* wtot)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int begin = t * kPerThread;
    DD local{0.0, 0.0};
    DD mine[kPerThread];
    for (int i = 0; i < kPerThread; ++i) {
        const int k = begin + i;
        if (k < n) local = dd_add(local, DD{w[k], 0.0});
        mine[i] = local;
    }
    DD incl = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const DD o = dd_shfl_up(incl, off);
        if (lane >= off) incl = dd_add(o, incl);
    }
    __syncthreads();
    if (lane == 31) wtot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        DD v = lane < kWarps ? wtot[lane] : DD{0.0, 0.0};
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const DD o = dd_shfl_up(v, off);
            if (lane >= off) v = dd_add(o, v);
        }
        if (lane < kWarps) wtot[lane] = v;  // inclusive warp totals
    }
    __syncthreads();
    // exclusive prefix of this thread = (incl - local) within the warp + earlier warps
    DD before = dd_add(incl, DD{-local.hi, -local.lo});
    if (warp > 0) before = dd_add(wtot[warp - 1], before);
    for (int i = 0; i < kPerThread; ++i) {
        const int k = begin + i;
        if (k < n) {
            const DD c = dd_add(before, mine[i]);
            chi[k] = c.hi;
            clo[k] = c.lo;
        }
    }
    __syncthreads();
}

// Weighted-Estimates (inverse-variance weights, chi^2 per degree of freedom)
// and Check-Convergence over n recorded iterations; one thread.  Returns
// whether the result has converged.
static __device__ bool weigh_and_check(const double* hI, const double* hV, int n, double rel_tol, double abs_tol,
                                double* est, double* sigma, double* chi2_dof)
{
    int n_exact = 0;
    double exact_sum = 0.0;
    for (int i = 0; i < n; ++i)
        if (hV[i] == 0.0) { ++n_exact; exact_sum += hI[i]; }
    double I, sig, chi2 = 0.0;
    if (n_exact > 0) {
        I = exact_sum / n_exact;
        sig = 0.0;
    } else {
        double sw = 0.0, swi = 0.0;
        for (int i = 0; i < n; ++i) {
            const double w = 1.0 / hV[i];
            sw += w;
            swi += w * hI[i];
        }
        I = swi / sw;
        sig = sqrt(1.0 / sw);
        if (n > 1) {
            for (int i = 0; i < n; ++i) {
                const double z = hI[i] - I;
                chi2 += z * z / hV[i];
            }
            chi2 /= (double)(n - 1);
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
                                          double* scratch, int split = 1, double p = 0.0)
{
    double s0 = 0.0, s1 = 0.0;
    if (split > 1) {
        const int ncubes = nparts / split;
        const double q = ceil(p / split);
        for (int cb = threadIdx.x; cb < ncubes; cb += blockDim.x) {
            const double* v = part + 3 * (size_t)cb * split;
            const double K0 = v[0];
            double S1 = 0.0, S2 = 0.0;
            for (int k = 0; k < split; ++k) {
                const double n = fmin(q, fmax(p - q * k, 0.0));
                const double dK = v[3 * k] - K0;
                S2 += fma(dK, fma(n, dK, 2.0 * v[3 * k + 1]), v[3 * k + 2]);
                S1 += fma(n, dK, v[3 * k + 1]);
            }
            s0 += K0 + S1 / p;
            s1 += (S2 - S1 * S1 / p) / (p * (p - 1.0));
        }
    } else {
        for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
            s0 += part[3 * (size_t)b + 0];
            s1 += part[3 * (size_t)b + 1];
        }
    }
    s0 = block_sum(s0, scratch);
    s1 = block_sum(s1, scratch);
    if (threadIdx.x == 0) {
        const double I = s0 / m;
        const double V = s1 / (m * m);
        const int n = *r.n;
        if (n < r.cap) {
            r.hist_I[n] = I;
            r.hist_V[n] = V;
            *r.n = n + 1;
        }
        if (!isfinite(I) || !isfinite(V)) {
            *r.error = MCUBES_ENONFINITE;
            *r.done = 1;
        } else if (weigh_and_check(r.hist_I, r.hist_V, *r.n, r.rel_tol, r.abs_tol, r.estimate, r.sigma,
                                   r.chi2_dof)) {
            *r.converged = 1;
            *r.done = 1;
        }
        *r.it += 1;
    }
}

// Adjust-Bin-Bounds of one axis (Lepage 1978, as the paper's Alg. 2 cites):
// smooth the bin sums with their neighbours, normalise, compress with
// ((r - 1) / ln r)^alpha, then place the new right edges where the
// cumulative compressed weight reaches i / nb of its total, the weight of an
// old bin being spread evenly over it.  The cumulative weight and the
// targets are double-double, so an edge is exact to about 2^-104 of the total
// weight and the new bin widths keep full double precision.
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
    __shared__ double sW[kNbMax];
    __shared__ double sB[kNbMax];
    __shared__ double sLo[kNbMax];
    __shared__ double sBlo[kNbMax];
    __shared__ DD wtot[kWarps];
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
    double part = 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        double sm;
        if (k == 0) sm = (sC[0] + sC[1]) / 2.0;
        else if (k == nb - 1) sm = (sC[nb - 2] + sC[nb - 1]) / 2.0;
        else sm = (sC[k - 1] + sC[k] + sC[k + 1]) / 3.0;
        sW[k] = sm;
    }
    __syncthreads();
    // fixed-order total: contiguous chunks per thread, then the tree
    for (int i = 0; i < kPerThread; ++i) {
        const int k = threadIdx.x * kPerThread + i;
        if (k < nb) part += sW[k];
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
    // compression ((r - 1)/ln r)^alpha with the library's log/exp (their FP64
    // work is a few instructions; CUDA's log and pow cost ~100 on a pipe
    // that issues 2 per clock per SM, and one block runs an axis)
    const double inv_total = 1.0 / total;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        const double r = sW[k] * inv_total;
        double w;
        if (r <= 0.0) w = 0.0;
        else if (r == 1.0) w = 1.0;
        else {
            const double q = (r - 1.0) / fx::fx_log(r);
            w = alpha == 1.5 ? q * sqrt(q) : fx::fx_exp(alpha * fx::fx_log(q));
        }
        sW[k] = w;
    }
    __syncthreads();
    // sC, sLo = cumulative weight through bin k (double-double)
    dd_inclusive_scan(sW, sC, sLo, nb, wtot);
    const DD wsum{sC[nb - 1], sLo[nb - 1]};
    if (!(wsum.hi > 0.0) || !isfinite(wsum.hi)) {
        if (threadIdx.x == 0) {
            *error = MCUBES_ENONFINITE;
            *done = 1;
        }
        return;
    }
    double* out = grid;
    double* out_lo = grid_lo;
    for (int i = 1 + threadIdx.x; i < nb; i += blockDim.x) {
        const DD target = dd_div(dd_scale(wsum, (double)i), (double)nb);
        // first bin k whose cumulative weight through k reaches the target
        int lo = 0, hi = nb - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (dd_ge(DD{sC[mid], sLo[mid]}, target)) hi = mid; else lo = mid + 1;
        }
        const int k = lo;
        const DD before = k > 0 ? DD{sC[k - 1], sLo[k - 1]} : DD{0.0, 0.0};
        const DD rem = dd_add(target, DD{-before.hi, -before.lo});
        const DD left = k > 0 ? DD{sB[k - 1], sBlo[k - 1]} : DD{0.0, 0.0};
        const DD width = dd_add(DD{sB[k], sBlo[k]}, DD{-left.hi, -left.lo});
        double frac = (rem.hi + rem.lo) / sW[k];
        frac = fmin(fmax(frac, 0.0), 1.0);
        const DD e = dd_add(left, dd_scale(width, frac));
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
