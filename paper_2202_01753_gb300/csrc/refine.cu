// refine.cu -- per-iteration finalisation of a single integral on the
// device: the fixed-order reduction of the sampling launch's block partials,
// Adjust-Bin-Bounds (Alg. 2) as one block per axis (reading and clearing the
// pass's histogram, then rebuilding that axis's map cells), and
// Weighted-Estimates plus Check-Convergence (Alg. 2) as one more block.
// Keeping these on the GPU lets a whole iteration run without the host.
#include "refine_dev.cuh"

namespace mc {

namespace {

using namespace refine_detail;

__global__ void __launch_bounds__(kRefineThreads) refine_kernel(const __grid_constant__ RefineArgs a)
{
    __shared__ double scratch[33];
    if (!*(volatile const int*)&a.st->active) return;  // iteration skipped after convergence
    DevState* st = a.st;
    const int nrebin = a.adjust ? a.hist_d : 0;
    if ((int)blockIdx.x == nrebin) {
        const IterRecord r{&st->it, &st->done, &st->error, &st->n, &st->converged, &st->estimate, &st->sigma,
                           &st->chi2_dof, st->hist_I, st->hist_V, kItMax, st->rel_tol, st->abs_tol};
        finalize_iteration(a.part, a.nblocks, a.m, r, scratch, a.split, a.p);
    } else {
        const int ax = blockIdx.x;
        const size_t off = (size_t)ax * a.nb;
        const int rows = a.hist_d == a.d ? 1 : a.d;  // m-Cubes1D: axis 0's edges go to every axis
        rebin_axis(a.hist_acc + off, 0, 1, false, a.nb, a.alpha, a.grid + off, a.grid_lo + off, a.hist + off,
                   &st->error, &st->done, scratch, rows);
        // rebin_axis read the row before its first barrier: clear it for the next pass
        for (int k = threadIdx.x; k < a.nb; k += blockDim.x) a.hist_acc[off + k] = 0.0;
        if (a.cells_g) {
            __syncthreads();  // the block's new edges are in global memory
            const double inv_g = 1.0 / (double)a.g;
            for (int r = 0; r < rows; ++r) {
                const int j = ax + r;
                const double* row = a.grid + (size_t)j * a.nb;
                const double* row_lo = a.grid_lo + (size_t)j * a.nb;
                for (int k = threadIdx.x; k < a.nb; k += blockDim.x) {
                    const size_t i = (size_t)j * a.nb + k;
                    if (a.mixed)
                        static_cast<float2*>(a.cells_g)[i] = map_cell_f32(row, row_lo, k, a.lo[j], a.scale[j], a.nb);
                    else
                        static_cast<double2*>(a.cells_g)[i] = map_cell_f64(row, row_lo, k, a.lo[j], a.scale[j], inv_g);
                }
            }
        }
    }
}

// Sums of one sampling pass over a cube range (no state change): block
// d (or 0) adds the partial sums, blocks 0..d-1 copy the histogram rows out
// of the accumulator and clear them (d is the number of axes with a
// histogram).
__global__ void __launch_bounds__(kRefineThreads)
reduce_range_kernel(const double* part, double* hist_acc, int nblocks, int d, int nb, int adjust,
                    double* out_sums, double* out_hist)
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
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        const size_t i = (size_t)ax * nb + k;
        out_hist[i] = hist_acc[i];
        hist_acc[i] = 0.0;
    }
}

// Map cells of the whole grid (set-up, and after the grid is replaced).
__global__ void cells_kernel(const double* grid, const double* grid_lo, CellBox box, int d, int nb, void* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d * nb) return;
    const int j = i / nb, k = i - j * nb;
    const double* row = grid + (size_t)j * nb;
    const double* row_lo = grid_lo + (size_t)j * nb;
    if (box.mixed) static_cast<float2*>(out)[i] = map_cell_f32(row, row_lo, k, box.lo[j], box.scale[j], nb);
    else static_cast<double2*>(out)[i] = map_cell_f64(row, row_lo, k, box.lo[j], box.scale[j], 1.0 / (double)box.g);
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
    const int blocks = (a.adjust ? a.hist_d : 0) + 1;
    refine_kernel<<<blocks, kRefineThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_reduce_range(const double* part, double* hist_acc, int nblocks, int d, int nb, int adjust,
                                double* out_sums, double* out_hist, cudaStream_t s)
{
    const int blocks = (adjust ? d : 0) + 1;
    reduce_range_kernel<<<blocks, kRefineThreads, 0, s>>>(part, hist_acc, nblocks, d, nb, adjust, out_sums,
                                                          out_hist);
    return cudaGetLastError();
}

cudaError_t launch_cells(const double* grid, const double* grid_lo, const CellBox& box, int d, int nb, void* out,
                         cudaStream_t s)
{
    const int n = d * nb;
    cells_kernel<<<(n + 255) / 256, 256, 0, s>>>(grid, grid_lo, box, d, nb, out);
    return cudaGetLastError();
}

cudaError_t launch_init_grid(double* grid, double* grid_lo, int d, int nb, cudaStream_t s)
{
    const int n = d * nb;
    init_grid_kernel<<<(n + 255) / 256, 256, 0, s>>>(grid, grid_lo, d, nb);
    return cudaGetLastError();
}

}  // namespace mc
