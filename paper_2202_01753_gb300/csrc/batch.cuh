// batch.cuh -- the persistent batched sampling kernels: one launch per class
// of integrals (integrand family x dimension) samples one
// iteration of every live integral of that class.  The host lays the class's
// live integrals' samples end to end and cuts that line into one equal,
// cube-aligned chunk per block; a block therefore samples a few segments
// (runs of cubes of one integral each), in order.  Per segment it stages that
// integral's grid and family constants in shared memory, samples with the
// same per-sample code as the single-integral kernel (vsample.cuh), and
// writes the segment's partial sums and, in adjusting iterations, its
// partial histogram.  The refinement launch (batch.cu) reduces an integral's
// segments in their fixed order.  One kernel per class keeps each one fully
// inlined with the register budget of the single-integral kernel.
#pragma once

#include "vsample.cuh"

namespace mc {

// One kernel per (family, dimension D): every segment it samples belongs to
// an integral of that dimension.  Registers are bounded as for the
// single-integral kernel of the same family and axis count (3 or 4 resident
// blocks per SM), so that more blocks of the concurrently running classes
// fit on an SM.
template <int FAM, bool MIXED, int D>
__global__ void __launch_bounds__(kVsThreads, vsample_min_blocks<FAM, MIXED, (D + 3) / 4>())
vsample_batch_kernel(const __grid_constant__ BatchArgs a)
{
    constexpr int NB4 = (D + 3) / 4;
    if constexpr (FAM == MCUBES_F_COSMO6 && D != 6) {
        return;  // six axes only: never launched
    } else {
    using Cell = typename Prec<MIXED>::Cell;
    using HT = typename Prec<MIXED>::H;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[3][kVsThreads / 32];
    __shared__ __align__(16) BatchDesc sd;

    const uint32_t s_begin = a.blk_seg[blockIdx.x], s_end = a.blk_seg[blockIdx.x + 1];
    for (uint32_t si = s_begin; si < s_end; ++si) {
        const BatchSeg seg = a.segs[si];
        __syncthreads();  // the previous segment is done with sd, cells and hist
        {
            const uint32_t* src = reinterpret_cast<const uint32_t*>(a.desc + seg.slot);
            uint32_t* dst = reinterpret_cast<uint32_t*>(&sd);
            for (uint32_t i = threadIdx.x; i < sizeof(BatchDesc) / 4; i += blockDim.x) dst[i] = src[i];
        }
        __syncthreads();
        // an integral that finished in an earlier iteration of this step (a
        // step may run several) is skipped; only the refinement changes the state
        const BatchState& B = a.st[seg.slot];
        if (B.done || (int)B.it >= sd.itmax) continue;
        // this iteration adjusts while it < ita (a step's iterations may cross
        // ita); the refinement reads the flag back
        const bool adjust = seg.adjust && (int)B.it < sd.ita;
        if (threadIdx.x == 0) a.segs[si].adjust = adjust ? 1u : 0u;
        constexpr uint32_t d = D;
        const uint32_t nb = sd.nb;
        Cell* cells = reinterpret_cast<Cell*>(smem);
        HT* hist = reinterpret_cast<HT*>(smem + cell_bytes(MIXED) * d * nb);
        if (adjust) stage_cells<MIXED, true>(cells, hist, sd.cells, d, nb, d);
        else stage_cells<MIXED, false>(cells, hist, sd.cells, d, nb, d);
        __syncthreads();

        const BatchView v{d,        nb,           sd.g,     sd.gmagic,         sd.key0,          sd.key1, d,
                          sd.jac0,  sd.phi_scale_f, sd.inv_p, sd.inv_var_den, sd.inv_p_f, sd.inv_var_den_f, 0u,
                          sd.fam};
        const uint32_t it = B.it;
        CubeSums acc;
        if (adjust)
            sample_cubes<FAM, MIXED, true, NB4, D>(v, cells, hist, seg.c0, seg.c1 - seg.c0, seg.perm_k, 0, 1, it,
                                                sd.lanes, sd.p, acc);
        else
            sample_cubes<FAM, MIXED, false, NB4, D>(v, cells, hist, seg.c0, seg.c1 - seg.c0, seg.perm_k, 0, 1, it,
                                                 sd.lanes, sd.p, acc);
        block_write_sums(acc, red, a.seg_part + 3 * (size_t)si);
        if (adjust) {
            __syncthreads();
            HT* out = reinterpret_cast<HT*>(a.seg_hist) + seg.hist_off;
            for (uint32_t i = threadIdx.x; i < d * nb; i += blockDim.x) out[i] = hist[i];
        }
    }
    }
}

template <int FAM, bool MIXED>
inline auto vsample_batch_kernel_ptr(int d)
{
    using K = void (*)(BatchArgs);
    switch (d) {
    case 1: return (K)vsample_batch_kernel<FAM, MIXED, 1>;
    case 2: return (K)vsample_batch_kernel<FAM, MIXED, 2>;
    case 3: return (K)vsample_batch_kernel<FAM, MIXED, 3>;
    case 4: return (K)vsample_batch_kernel<FAM, MIXED, 4>;
    case 5: return (K)vsample_batch_kernel<FAM, MIXED, 5>;
    case 6: return (K)vsample_batch_kernel<FAM, MIXED, 6>;
    case 7: return (K)vsample_batch_kernel<FAM, MIXED, 7>;
    case 8: return (K)vsample_batch_kernel<FAM, MIXED, 8>;
    case 9: return (K)vsample_batch_kernel<FAM, MIXED, 9>;
    case 10: return (K)vsample_batch_kernel<FAM, MIXED, 10>;
    case 11: return (K)vsample_batch_kernel<FAM, MIXED, 11>;
    default: return (K)vsample_batch_kernel<FAM, MIXED, 12>;
    }
}

template <int FAM>
cudaError_t launch_vsample_batch_family(bool mixed, int d, const BatchArgs& a, int grid, size_t smem,
                                        cudaStream_t s)
{
    auto k = mixed ? vsample_batch_kernel_ptr<FAM, true>(d) : vsample_batch_kernel_ptr<FAM, false>(d);
    cudaError_t e = raise_smem_limit((const void*)k, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kVsThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int FAM>
cudaError_t vsample_batch_occupancy_family(bool mixed, int d, size_t smem, int* blocks)
{
    auto k = mixed ? vsample_batch_kernel_ptr<FAM, true>(d) : vsample_batch_kernel_ptr<FAM, false>(d);
    cudaError_t e = raise_smem_limit((const void*)k, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, kVsThreads, smem);
}

}  // namespace mc

// Instantiates a family's batched kernels and their launchers
// (launch_vsample_batch_<name>, vsample_batch_occupancy_<name>).
#define MC_INSTANTIATE_BATCH_FAMILY(FAM, NAME)                                                        \
    namespace mc {                                                                                    \
    cudaError_t launch_vsample_batch_##NAME(bool mixed, int d, const BatchArgs& a, int grid,          \
                                            size_t smem, cudaStream_t s)                              \
    {                                                                                                 \
        return launch_vsample_batch_family<FAM>(mixed, d, a, grid, smem, s);                          \
    }                                                                                                 \
    cudaError_t vsample_batch_occupancy_##NAME(bool mixed, int d, size_t smem, int* blocks)           \
    {                                                                                                 \
        return vsample_batch_occupancy_family<FAM>(mixed, d, smem, blocks);                           \
    }                                                                                                 \
    }
