// mc_internal.h -- structures shared by the host driver and the kernels of
// the GB300 m-Cubes library.  Not part of the public ABI (include/mcubes.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "mcubes.h"

namespace mc {

constexpr int kDMax = MCUBES_DMAX;
constexpr int kNbMax = MCUBES_NBMAX;
constexpr int kParMax = MCUBES_PARAMS_MAX;
constexpr int kItMax = MCUBES_ITMAX_MAX;
constexpr int kVsThreads = 256;    // sampling block size (8 warps); batched kernels
constexpr int kVsThreadsMax = 1024; // largest block of a single-integral sampling kernel

// Block size of a single-integral sampling kernel.  Its warps hide the
// latency of a serial chain per sample, so resident warps count: the
// registers a kernel needs bound them (65536 per SM), and a block size that
// fills that bound beats 256-thread blocks whose count per SM is capped by
// shared memory (three blocks of the FP64 six-axis grid and histogram).
// The FP64 six-axis kernel (62 registers) runs one block of 1024 threads per
// SM: measured 8.19 ms per 1e8-call pass against 8.39 (2 x 512), 8.54
// (2 x 448), 8.94 (3 x 320), 8.92 (3 x 288) and 8.79 ms (3 x 256).
constexpr int kCosmo6Threads = 1024;
__host__ __device__ constexpr int vsample_threads(int family, bool mixed, int d)
{
    return (family == MCUBES_F_COSMO6 && !mixed && d == 6) ? kCosmo6Threads : kVsThreads;
}
constexpr int kRefineThreads = 512;

// Shared-memory bytes per bin of the sampling kernels: a grid cell (left
// edge, nb * width) in double or single precision, and a histogram entry.
__host__ __device__ constexpr size_t cell_bytes(bool mixed) { return mixed ? 8 : 16; }
__host__ __device__ constexpr size_t hist_bytes(bool mixed) { return mixed ? 4 : 8; }

// Per-integral state kept on the device across iterations, so that the whole
// iteration loop (sample -> refine -> weight -> converge) runs without the
// host.  One instance per single-integral context.
struct DevState {
    uint32_t it;        // iteration index of the next sampling pass
    int done;           // converged or failed: further iterations are skipped
    int active;         // set by the sampling launch: this iteration ran
    int error;          // mcubes_status of a failure seen on the device
    int n;              // iterations recorded
    int converged;
    double estimate, sigma, chi2_dof;
    double rel_tol, abs_tol;
    double hist_I[kItMax];
    double hist_V[kItMax];
};

// One interpolation table as the kernels read it (TABLE family): values in
// double (v) and single (vf) precision, knots i at lo + i / s.
struct TableDesc {
    const double* v;
    const float* vf;
    int ndim, n0, n1, pad;
    double lo0, hi0, s0, lo1, hi1, s1;   // s = (n - 1) / (hi - lo)
    double los0, los1;                    // lo * s (rounded): u = (x - lo) s as fma(x, s, -lo s)
    float lo0f, hi0f, s0f, lo1f, hi1f, s1f;
};

constexpr int kTabFactorsMax = 10;

// Integrand constants in the form the kernels use (derived on the host from
// the public params blob, see integrand_prepare in capi.cu).
struct FamParams {
    double c[kParMax];
    float cf[kParMax];
    // TABLE family: factor q reads table tid[q] at axes a[q] (and b[q] >= 0)
    int nf;
    int tid[kTabFactorsMax], ta[kTabFactorsMax], tb[kTabFactorsMax];
    const TableDesc* tabs;   // device array of the context's tables
};

// Arguments of one sampling launch (Alg. 3).  Passed by value as a
// __grid_constant__ kernel parameter: indices known at compile time become
// constant-bank operands.
struct VsArgs {
    const double* grid;       // [d][nb] right edges, unit coordinates (double-double: high parts)
    const double* grid_lo;    // [d][nb] low parts
    double* part;             // [gridDim][3]: sum of cube means, of their variances, of |means|
    const void* cells_g;      // [d][nb] map cells of the current grid (double2 or float2), or null: build
                              // them from grid/grid_lo in every block
    double* hist_acc;         // [hist_d][nb] sums of F^2 of this pass: zero before an adjusting launch;
                              // every block adds its shared-memory histogram once (global reductions)
    DevState* st;             // iteration state; nullptr -> use it_fixed and always run
    uint32_t it_fixed;
    uint32_t d, nb, g, gmagic;  // gmagic = floor((2^32-1)/g)
    uint32_t p, lanes;          // samples per cube, threads per cube (power of two <= 32)
    uint32_t hist_d;            // axes with a histogram: d, or 1 for m-Cubes1D (hist_acc is [hist_d][nb])
    uint32_t split;             // > 1: blocks per cube (cube-split mode: gridDim = cubes * split, part holds
                                // each block's shifted sums (K, S1, S2) of its slice of one cube)
    uint64_t cube_begin, cube_end;
    uint64_t perm_k;          // cube order: logical i -> cube_begin + (i perm_k mod n), gcd(perm_k, n) = 1
    uint32_t rk[10][2];       // Philox round keys (key + r * Weyl constants)
    double lo[kDMax];
    double scale[kDMax];      // hi - lo
    double jac0;              // (g nb)^d: FP64 cells hold width / g, so J = jac0 prod(cell widths)
    float phi_scale_f;        // 1 / (g nb): mixed cells hold nb width, so x = left + (nb width)(g phi)/(g nb)
    float nb_f;
    double inv_p, inv_var_den;     // 1/p and 1/(p (p-1)) of the cube moments (Alg. 3 UpdateVariance)
    float inv_p_f, inv_var_den_f;  // the same in single precision (mixed)
    uint32_t want_abs;             // part[2] (sums of |cube mean|) wanted: the sampling-pass calls
    FamParams fam;
};

// ---------------------------------------------------------------------------
// Batched iterations (many independent integrals per launch)
// ---------------------------------------------------------------------------

// One resident integral of a batch, as the batched kernels read it.
struct BatchDesc {
    uint32_t d, nb, g, gmagic;
    uint32_t p, lanes;
    uint32_t key0, key1;        // Philox key = the integral's own seed
    int family, ita, itmax, mixed;
    uint64_t m;
    double jac0;                // (g nb)^d
    double inv_p, inv_var_den;  // 1/p and 1/(p (p-1)) of the cube moments
    float phi_scale_f;          // 1 / (g nb)
    float inv_p_f, inv_var_den_f;
    float pad2;
    double lo[kDMax];
    double scale[kDMax];
    FamParams fam;
    double* grid;               // [d][nb] edge high parts, then [d][nb] low parts
    void* cells;                // [d][nb] map cells of the grid (double2 in FP64, float2 in mixed), rebuilt
                                // by the refinement after each rebin
    double* hist;               // [d][nb] histogram of the last adjusting iteration
    double* hist_I;             // [itmax] iteration estimates
    double* hist_V;             // [itmax] iteration variances
    double rel_tol, abs_tol;
};

// Per-integral iteration state of a batch (device).
struct BatchState {
    uint32_t it;
    int done, error, n, converged, pad;
    double estimate, sigma, chi2_dof;
};

// A run of cubes [c0, c1) of one integral, sampled by one block.
struct BatchSeg {
    uint32_t slot;
    uint32_t adjust;            // host: adjusting at the step's first iteration (the histogram space is
                                // reserved); device: whether this iteration adjusts
    uint64_t c0, c1;
    uint64_t perm_k;            // cube order within the segment (see sample_cubes)
    uint64_t hist_off;          // element offset of the segment's partial histogram
};

struct BatchArgs {
    const BatchDesc* desc;
    const BatchState* st;
    BatchSeg* segs;             // the sampling launch sets each segment's adjust for this iteration
    const uint32_t* blk_seg;    // block b samples segments [blk_seg[b], blk_seg[b+1]) (this class's table)
    double* seg_part;           // [segment][3] partial sums
    void* seg_hist;             // partial histograms (float in mixed, double in fp64)
};

struct BatchRefineArgs {
    const BatchDesc* desc;
    BatchState* st;
    const uint32_t* live;       // [capacity]: slot of live integral j
    const uint32_t* live_seg;   // [capacity + 1]: live integral j owns segments [live_seg[j], live_seg[j+1])
    const uint32_t* nlive;      // device scalar
    const BatchSeg* segs;
    const double* seg_part;
    const void* seg_hist;
    int hist_is_float;
    double alpha;
};

// Batched kernels are instantiated per class: family x dimension (an exact
// axis count unrolls the per-axis loops without guards).
constexpr int kNumClasses = MCUBES_F_TABLE * kDMax;  // families with batched kernels (not TABLE)
__host__ __device__ constexpr int batch_class(int family, int d) { return family * kDMax + d - 1; }
cudaError_t launch_vsample_batch(int cls, bool mixed, const BatchArgs& a, int grid, size_t smem, cudaStream_t s);
cudaError_t vsample_batch_occupancy(int cls, bool mixed, size_t smem, int* blocks_per_sm);
cudaError_t launch_refine_batch(const BatchRefineArgs& a, int capacity, int rows, cudaStream_t s);
cudaError_t launch_init_slots(const BatchDesc* desc, BatchState* st, const uint32_t* slots, int count,
                              cudaStream_t s);

struct RefineArgs {
    double* grid;             // [d][nb] edge high parts, updated in place by the rebin blocks
    double* grid_lo;          // [d][nb] edge low parts
    double* hist;             // [d][nb] reduced histogram (written for read-back)
    const double* part;       // [nblocks][3]
    double* hist_acc;         // [hist_d][nb] histogram of the sampling pass; read, then cleared
    void* cells_g;            // [d][nb] map cells, rebuilt for every rebinned axis (null: none kept)
    double lo[kDMax], scale[kDMax];
    uint32_t g;
    int mixed;
    DevState* st;
    int nblocks, d, nb, adjust;
    int hist_d;               // axes with a histogram: d, or 1 (m-Cubes1D: axis 0's new edges go to every axis)
    int split;                // > 1: part holds (K, S1, S2) per block, split blocks per cube
    double p;                 // samples per cube
    double alpha;
    double m;                 // number of cubes
};

// The box and format of the map cells (cells_kernel).
struct CellBox {
    double lo[kDMax], scale[kDMax];
    uint32_t g;
    int mixed;
};
cudaError_t launch_cells(const double* grid, const double* grid_lo, const CellBox& box, int d, int nb, void* out,
                         cudaStream_t s);

// Launchers (one per integrand family translation unit).
cudaError_t launch_vsample(int family, bool mixed, bool adjust, const VsArgs& a, int grid,
                           size_t smem, cudaStream_t s);
size_t vsample_smem_bytes(bool mixed, bool adjust, int d, int nb, int hist_d);
cudaError_t vsample_occupancy(int family, bool mixed, bool adjust, int d, size_t smem, int* blocks_per_sm);
uint64_t cube_permutation(uint64_t n);
// Raises a kernel's dynamic shared-memory limit on the current device to at
// least smem bytes (never lowers it, so that contexts of different sizes can
// share a kernel); a host-side record skips the driver call when the limit
// is already high enough.
cudaError_t raise_smem_limit(const void* kernel, size_t smem);
double jacobian_scale(long long g, long long nb, int d);  // (g nb)^d
double family_jac_factor(int id, const FamParams& fp);    // an FP64 family's constant factor
struct MomentScales {
    double inv_p, inv_var_den;
    float inv_p_f, inv_var_den_f;
};
MomentScales moment_scales(long long p);  // 1/p, 1/(p (p-1)), p >= 2
template <class T> void set_moment_scales(T& a, long long p)
{
    const MomentScales m = moment_scales(p);
    a.inv_p = m.inv_p;
    a.inv_var_den = m.inv_var_den;
    a.inv_p_f = m.inv_p_f;
    a.inv_var_den_f = m.inv_var_den_f;
}

cudaError_t launch_refine(const RefineArgs& a, cudaStream_t s);
cudaError_t launch_reduce_range(const double* part, double* hist_acc, int nblocks, int d, int nb, int adjust,
                                double* out_sums, double* out_hist, cudaStream_t s);
cudaError_t launch_init_grid(double* grid, double* grid_lo, int d, int nb, cudaStream_t s);
// Sums nranks partials ([nranks][len], rank order) element by element in rank
// order: the first MCUBES_SHARD_HEAD sums go to part[0..], the rest to hist.
cudaError_t launch_combine_shards(const double* gathered, int nranks, int len, double* part, double* hist,
                                  cudaStream_t s);

}  // namespace mc
