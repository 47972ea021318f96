// refine.cu -- per-iteration finalisation of a single integral on the
// device: the fixed-order reduction of the sampling launch's block partials,
// Adjust-Bin-Bounds (Alg. 2) as one block per axis (reading and clearing the
// pass's histogram, then rebuilding that axis's map cells), and
// Weighted-Estimates plus Check-Convergence (Alg. 2) as one more block.
// Keeping these on the GPU lets a whole iteration run without the host.
#include <cooperative_groups.h>

#include "refine_dev.cuh"

namespace mc {

namespace cg = cooperative_groups;

namespace {

using namespace refine_detail;

constexpr int kRebinCtas = 4;  // blocks (SMs) per rebinned axis: one thread-block cluster

// Adjust-Bin-Bounds of axis ax by the kRebinCtas blocks of one thread-block
// cluster: every block loads the axis and computes the smoothed total (the
// same value in each), block `rank` compresses its chunk of the bins into
// shared memory, every block gathers the whole axis's weights through the
// cluster's distributed shared memory and scans them (exact integers: the
// same sums in each), then computes the new edges and map cells of its chunk.
// The FP64 work per bin (the compression, the fraction and the double-double
// edge) is spread over kRebinCtas SMs instead of one.
static __device__ void rebin_axis_cluster(const RefineArgs& a, int ax, int rank, cg::cluster_group& cluster,
                                          double* scratch)
{
    constexpr int R = kRebinCtas;
    constexpr int kChunkMax = (kNbMax + R - 1) / R;
    __shared__ __align__(16) unsigned char s_raw[sizeof(u128) * kNbMax];  // sC, then sCum
    __shared__ double sB[kNbMax];
    __shared__ double sBlo[kNbMax];
    __shared__ u128 sWq[kChunkMax];
    __shared__ double sEh[kChunkMax];
    __shared__ double sEl[kChunkMax];
    __shared__ u128 wtot[kWarps];
    double* sC = reinterpret_cast<double*>(s_raw);
    u128* sCum = reinterpret_cast<u128*>(s_raw);
    DevState* st = a.st;
    const int nb = a.nb;
    const size_t off = (size_t)ax * nb;
    const int rows = a.hist_d == a.d ? 1 : a.d;  // m-Cubes1D: axis 0's edges go to every axis
    const int chunk = (nb + R - 1) / R;
    const int k0 = rank * chunk, k1 = min(nb, k0 + chunk);
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        const double c = a.hist_acc[off + k];
        sC[k] = c;
        if (rank == 0) a.hist[off + k] = c;
        sB[k] = a.grid[off + k];
        sBlo[k] = a.grid_lo[off + k];
    }
    __syncthreads();
    double part = 0.0;
    for (int i = 0; i < kPerThread; ++i) {
        const int k = threadIdx.x * kPerThread + i;
        if (k < nb) part += smoothed3(sC, k, nb);  // fixed order, as in rebin_axis
    }
    const double total = block_sum(part, scratch);  // the same in every block of the cluster
    const bool finite = isfinite(total);
    const bool rebin = finite && total > 0.0;      // else: no information (or an error), grid unchanged
    if (!finite && rank == 0 && threadIdx.x == 0) {
        st->error = MCUBES_ENONFINITE;
        st->done = 1;
    }
    if (rebin) {
        const double inv_total = 1.0 / total;
        for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x)
            sWq[k - k0] = compressed_weight(smoothed3(sC, k, nb), inv_total, a.alpha);
    }
    cluster.sync();  // every block has read the histogram row and the grid, and written its weights
    for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) a.hist_acc[off + k] = 0.0;  // for the next pass
    if (!rebin) return;  // the same in every block; no shared memory is read from here on
    u128 v[kPerThread];
#pragma unroll
    for (int i = 0; i < kPerThread; ++i) {
        const int k = threadIdx.x * kPerThread + i;
        const int owner = k / chunk;
        v[i] = k < nb ? cluster.map_shared_rank(sWq, owner)[k - owner * chunk] : (u128)0;
    }
    cluster.sync();  // every block has its copy: no block reads another's weights any more
    u128_inclusive_scan(v, sCum, nb, wtot);  // sC is no longer used: sCum takes its place
    const u128 W = sCum[nb - 1];
    if (W == 0) {
        if (rank == 0 && threadIdx.x == 0) {
            st->error = MCUBES_ENONFINITE;
            st->done = 1;
        }
        return;
    }
    for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const DD e = k < nb - 1 ? rebin_edge(k + 1, nb, W, sCum, sB, sBlo) : DD{1.0, 0.0};
        sEh[k - k0] = e.hi;
        sEl[k - k0] = e.lo;
        for (int r = 0; r < rows; ++r) {
            a.grid[off + (size_t)r * nb + k] = e.hi;
            a.grid_lo[off + (size_t)r * nb + k] = e.lo;
        }
    }
    if (!a.cells_g) return;
    cluster.sync();  // every block's new edges are in its shared memory
    const double inv_g = 1.0 / (double)a.g;
    for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const DD right{sEh[k - k0], sEl[k - k0]};
        DD left{0.0, 0.0};
        if (k > k0) left = DD{sEh[k - k0 - 1], sEl[k - k0 - 1]};
        else if (k > 0) left = DD{cluster.map_shared_rank(sEh, rank - 1)[chunk - 1],
                                  cluster.map_shared_rank(sEl, rank - 1)[chunk - 1]};
        for (int r = 0; r < rows; ++r) {
            const int j = ax + r;
            double xl, xw;
            map_cell_edges(left, right, a.lo[j], a.scale[j], &xl, &xw);
            const size_t i = (size_t)j * nb + k;
            if (a.mixed) static_cast<float2*>(a.cells_g)[i] = make_float2((float)xl, (float)(xw * (double)nb));
            else static_cast<double2*>(a.cells_g)[i] = make_double2(xl, xw * inv_g);
        }
    }
    cluster.sync();  // no block leaves while its neighbour reads its edges
}

// One iteration's finalisation: cluster c < nrebin rebins axis c (see
// rebin_axis_cluster), the last cluster's first block reduces the partials,
// records the iteration and weighs all of them.
__global__ void __cluster_dims__(kRebinCtas, 1, 1) __launch_bounds__(kRefineThreads)
refine_kernel(const __grid_constant__ RefineArgs a)
{
    __shared__ double scratch[33];
    if (!*(volatile const int*)&a.st->active) return;  // iteration skipped after convergence: the whole grid
    cg::cluster_group cluster = cg::this_cluster();
    const int c = (int)(blockIdx.x / kRebinCtas);
    const int rank = (int)cluster.block_rank();
    const int nrebin = a.adjust ? a.hist_d : 0;
    if (c == nrebin) {
        if (rank != 0) return;
        DevState* st = a.st;
        const IterRecord r{&st->it, &st->done, &st->error, &st->n, &st->converged, &st->estimate, &st->sigma,
                           &st->chi2_dof, st->hist_I, st->hist_V, kItMax, st->rel_tol, st->abs_tol};
        finalize_iteration(a.part, a.nblocks, a.m, r, a.split, a.p);
        return;
    }
    rebin_axis_cluster(a, c, rank, cluster, scratch);
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

// Rank-order sum of gathered shard partials (mcubes_shard_finish): one
// thread per element, the ranks added in order 0, 1, ... so that every rank
// that combines the same gathered array gets the same bits.
__global__ void combine_shards_kernel(const double* gathered, int nranks, int len, double* part, double* hist)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    double s = gathered[i];
    for (int r = 1; r < nranks; ++r) s += gathered[(size_t)r * len + i];
    if (i < MCUBES_SHARD_HEAD) part[i] = s;
    else hist[i - MCUBES_SHARD_HEAD] = s;
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
    const int clusters = (a.adjust ? a.hist_d : 0) + 1;
    refine_kernel<<<clusters * kRebinCtas, kRefineThreads, 0, s>>>(a);
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

cudaError_t launch_combine_shards(const double* gathered, int nranks, int len, double* part, double* hist,
                                  cudaStream_t s)
{
    combine_shards_kernel<<<(len + 255) / 256, 256, 0, s>>>(gathered, nranks, len, part, hist);
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
