// refine.cu -- per-iteration finalisation on the device: the fixed-order
// reduction of the sampling launch's block partials, Adjust-Bin-Bounds
// (Alg. 2) as one block per axis, and Weighted-Estimates plus
// Check-Convergence (Alg. 2) as one more block.  Keeping these on the GPU
// lets a whole iteration run without the host.
#include <cmath>

#include "mc_device.cuh"

namespace mc {

namespace {

constexpr int kWarps = kRefineThreads / 32;
constexpr int kPerThread = (kNbMax + kRefineThreads - 1) / kRefineThreads;

// Deterministic block sum (each thread's value added in a fixed tree).
__device__ double block_sum(double v, double* scratch)
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

__device__ __forceinline__ DD dd_shfl_up(DD v, int off)
{
    return DD{__shfl_up_sync(0xffffffffu, v.hi, off), __shfl_up_sync(0xffffffffu, v.lo, off)};
}

// Inclusive double-double prefix sum of w[0..n) into (chi, clo), fixed
// order: each thread adds kPerThread consecutive values, the thread totals
// are scanned by warp shuffles and then across warps.
__device__ void dd_inclusive_scan(const double* w, double* chi, double* clo, int n, DD* wtot)
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
// and Check-Convergence over the recorded iterations; one thread.
__device__ void weigh_and_check(DevState* st)
{
    const int n = st->n;
    int n_exact = 0;
    double exact_sum = 0.0;
    for (int i = 0; i < n; ++i)
        if (st->hist_V[i] == 0.0) { ++n_exact; exact_sum += st->hist_I[i]; }
    double I, sig, chi2 = 0.0;
    if (n_exact > 0) {
        I = exact_sum / n_exact;
        sig = 0.0;
    } else {
        double sw = 0.0, swi = 0.0;
        for (int i = 0; i < n; ++i) {
            const double w = 1.0 / st->hist_V[i];
            sw += w;
            swi += w * st->hist_I[i];
        }
        I = swi / sw;
        sig = sqrt(1.0 / sw);
        if (n > 1) {
            for (int i = 0; i < n; ++i) {
                const double z = st->hist_I[i] - I;
                chi2 += z * z / st->hist_V[i];
            }
            chi2 /= (double)(n - 1);
        }
    }
    st->estimate = I;
    st->sigma = sig;
    st->chi2_dof = chi2;
    const double tol = fmax(st->abs_tol, st->rel_tol * fabs(I));
    if (n >= 2 && sig <= tol) {
        st->converged = 1;
        st->done = 1;
    }
}

__device__ void finalize_block(const RefineArgs& a, double* scratch)
{
    double s0 = 0.0, s1 = 0.0;
    for (int b = threadIdx.x; b < a.nblocks; b += blockDim.x) {
        s0 += a.part[3 * (size_t)b + 0];
        s1 += a.part[3 * (size_t)b + 1];
    }
    s0 = block_sum(s0, scratch);
    s1 = block_sum(s1, scratch);
    if (threadIdx.x == 0) {
        DevState* st = a.st;
        const double I = s0 / a.m;
        const double V = s1 / (a.m * a.m);
        const int n = st->n;
        if (n < kItMax) {
            st->hist_I[n] = I;
            st->hist_V[n] = V;
            st->n = n + 1;
        }
        if (!isfinite(I) || !isfinite(V)) {
            st->error = MCUBES_ENONFINITE;
            st->done = 1;
        } else {
            weigh_and_check(st);
        }
        st->it += 1;
    }
}

// Adjust-Bin-Bounds of one axis (Lepage 1978, as the paper's Alg. 2 cites):
// smooth the bin sums with their neighbours, normalise, compress with
// ((r - 1) / ln r)^alpha, then place the new right edges where the
// cumulative compressed weight reaches i / nb of its total, the weight of an
// old bin being spread evenly over it.  The cumulative weight and the
// targets are double-double, so an edge is exact to about 2^-104 of the total
// weight and the new bin widths keep full double precision.
__device__ void rebin_block(const RefineArgs& a, int ax, double* scratch)
{
    __shared__ double sC[kNbMax];
    __shared__ double sW[kNbMax];
    __shared__ double sB[kNbMax];
    __shared__ double sLo[kNbMax];
    __shared__ double sBlo[kNbMax];
    __shared__ DD wtot[kWarps];
    const int nb = a.nb, d = a.d;
    const size_t stride = (size_t)d * nb;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        double acc = 0.0;
        if (a.hist_is_float) {
            const float* ph = static_cast<const float*>(a.part_hist) + (size_t)ax * nb + k;
            for (int b = 0; b < a.nblocks; ++b) acc += (double)ph[b * stride];
        } else {
            const double* ph = static_cast<const double*>(a.part_hist) + (size_t)ax * nb + k;
            for (int b = 0; b < a.nblocks; ++b) acc += ph[b * stride];
        }
        sC[k] = acc;
        a.hist[(size_t)ax * nb + k] = acc;
        sB[k] = a.grid[(size_t)ax * nb + k];
        sBlo[k] = a.grid_lo[(size_t)ax * nb + k];
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
            a.st->error = MCUBES_ENONFINITE;
            a.st->done = 1;
        }
        return;
    }
    if (total <= 0.0) return;  // no information on this axis: grid unchanged
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        const double r = sW[k] / total;
        double w;
        if (r <= 0.0) w = 0.0;
        else if (r == 1.0) w = 1.0;
        else w = pow((r - 1.0) / log(r), a.alpha);
        sW[k] = w;
    }
    __syncthreads();
    // sC, sLo = cumulative weight through bin k (double-double)
    dd_inclusive_scan(sW, sC, sLo, nb, wtot);
    const DD wsum{sC[nb - 1], sLo[nb - 1]};
    if (!(wsum.hi > 0.0) || !isfinite(wsum.hi)) {
        if (threadIdx.x == 0) {
            a.st->error = MCUBES_ENONFINITE;
            a.st->done = 1;
        }
        return;
    }
    double* out = a.grid + (size_t)ax * nb;
    double* out_lo = a.grid_lo + (size_t)ax * nb;
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
        out[i - 1] = e.hi;
        out_lo[i - 1] = e.lo;
    }
    if (threadIdx.x == 0) {
        out[nb - 1] = 1.0;
        out_lo[nb - 1] = 0.0;
    }
}

__global__ void __launch_bounds__(kRefineThreads) refine_kernel(const __grid_constant__ RefineArgs a)
{
    __shared__ double scratch[33];
    if (!*(volatile const int*)&a.st->active) return;  // iteration skipped after convergence
    const int nrebin = a.adjust ? a.d : 0;
    if ((int)blockIdx.x == nrebin) finalize_block(a, scratch);
    else rebin_block(a, blockIdx.x, scratch);
}

// Sums of one sampling pass over a cube range (no state change): block
// d (or 0) adds the partial sums, blocks 0..d-1 the histogram columns.
__global__ void __launch_bounds__(kRefineThreads)
reduce_range_kernel(const double* part, const void* part_hist, int hist_is_float, int nblocks, int d,
                    int nb, int adjust, double* out_sums, double* out_hist)
{
    __shared__ double scratch[33];
    const int nrebin = adjust ? d : 0;
    if ((int)blockIdx.x == nrebin) {
        double s[3] = {0.0, 0.0, 0.0};
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
            for (int q = 0; q < 3; ++q) s[q] += part[3 * (size_t)b + q];
        for (int q = 0; q < 3; ++q) {
            const double t = block_sum(s[q], scratch);
            if (threadIdx.x == 0) out_sums[q] = t;
        }
        return;
    }
    const int ax = blockIdx.x;
    const size_t stride = (size_t)d * nb;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        double acc = 0.0;
        if (hist_is_float) {
            const float* ph = static_cast<const float*>(part_hist) + (size_t)ax * nb + k;
            for (int b = 0; b < nblocks; ++b) acc += (double)ph[b * stride];
        } else {
            const double* ph = static_cast<const double*>(part_hist) + (size_t)ax * nb + k;
            for (int b = 0; b < nblocks; ++b) acc += ph[b * stride];
        }
        out_hist[(size_t)ax * nb + k] = acc;
    }
}

// Init-Bins (Alg. 2): nb equal bins per axis, right edges (k+1)/nb held as
// double-double (rounded value + rounded remainder), last edge exactly 1.
__global__ void init_grid_kernel(double* grid, double* grid_lo, int d, int nb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d * nb) return;
    const int k = i % nb;
    if (k == nb - 1) {
        grid[i] = 1.0;
        grid_lo[i] = 0.0;
        return;
    }
    const double hi = __ddiv_rn((double)(k + 1), (double)nb);
    const double rem = __fma_rn(-hi, (double)nb, (double)(k + 1));  // exact
    grid[i] = hi;
    grid_lo[i] = __ddiv_rn(rem, (double)nb);
}

}  // namespace

cudaError_t launch_refine(const RefineArgs& a, cudaStream_t s)
{
    const int blocks = (a.adjust ? a.d : 0) + 1;
    refine_kernel<<<blocks, kRefineThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_reduce_range(const double* part, const void* part_hist, int hist_is_float,
                                int nblocks, int d, int nb, int adjust, double* out_sums,
                                double* out_hist, cudaStream_t s)
{
    const int blocks = (adjust ? d : 0) + 1;
    reduce_range_kernel<<<blocks, kRefineThreads, 0, s>>>(part, part_hist, hist_is_float, nblocks, d,
                                                          nb, adjust, out_sums, out_hist);
    return cudaGetLastError();
}

cudaError_t launch_init_grid(double* grid, double* grid_lo, int d, int nb, cudaStream_t s)
{
    const int n = d * nb;
    init_grid_kernel<<<(n + 255) / 256, 256, 0, s>>>(grid, grid_lo, d, nb);
    return cudaGetLastError();
}

}  // namespace mc
