// batch.cuh -- the persistent batched sampling kernel: one launch samples one
// iteration of every live integral of a batch.  The host lays the live
// integrals' samples end to end and cuts that line into one equal,
// cube-aligned chunk per block; a block therefore samples a few segments
// (runs of cubes of one integral each), in order.  Per segment it stages that
// integral's grid and family constants in shared memory, samples with the
// same per-sample code as the single-integral kernel (vsample.cuh), and
// writes the segment's partial sums and, in adjusting iterations, its
// partial histogram.  The refinement launch (batch.cu) reduces an integral's
// segments in their fixed order.
#pragma once

#include "vsample.cuh"

namespace mc {

template <int FAM, bool MIXED>
__device__ __forceinline__ void batch_segment(const BatchView& v, const BatchDesc& sd,
                                              const typename Prec<MIXED>::Cell* cells,
                                              typename Prec<MIXED>::H* hist, const BatchSeg& seg, uint32_t it,
                                              CubeSums& acc)
{
    if (seg.adjust)
        sample_cubes<FAM, MIXED, true>(v, cells, hist, seg.c0, seg.c1 - seg.c0, 0, 1, it, sd.lanes, sd.p, acc);
    else
        sample_cubes<FAM, MIXED, false>(v, cells, hist, seg.c0, seg.c1 - seg.c0, 0, 1, it, sd.lanes, sd.p, acc);
}

template <bool MIXED>
__global__ void __launch_bounds__(kVsThreads) vsample_batch_kernel(const __grid_constant__ BatchArgs a)
{
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
        const uint32_t d = sd.d, nb = sd.nb;
        Cell* cells = reinterpret_cast<Cell*>(smem);
        HT* hist = reinterpret_cast<HT*>(smem + cell_bytes(MIXED) * d * nb);
        if (seg.adjust) stage_grid<MIXED, true>(cells, hist, sd.grid, sd.grid + d * nb, sd.lo, sd.scale, d, nb);
        else stage_grid<MIXED, false>(cells, hist, sd.grid, sd.grid + d * nb, sd.lo, sd.scale, d, nb);
        __syncthreads();

        const BatchView v{d, nb, sd.g, sd.gmagic, sd.key0, sd.key1, sd.phi_scale, sd.phi_scale_f, sd.fam};
        const uint32_t it = a.st[seg.slot].it;
        CubeSums acc;
        switch (sd.family) {
        case MCUBES_F_CONST: batch_segment<MCUBES_F_CONST, MIXED>(v, sd, cells, hist, seg, it, acc); break;
        case MCUBES_F_GAUSS: batch_segment<MCUBES_F_GAUSS, MIXED>(v, sd, cells, hist, seg, it, acc); break;
        case MCUBES_F_CORNER: batch_segment<MCUBES_F_CORNER, MIXED>(v, sd, cells, hist, seg, it, acc); break;
        case MCUBES_F_OSC: batch_segment<MCUBES_F_OSC, MIXED>(v, sd, cells, hist, seg, it, acc); break;
        case MCUBES_F_PRODPEAK: batch_segment<MCUBES_F_PRODPEAK, MIXED>(v, sd, cells, hist, seg, it, acc); break;
        case MCUBES_F_C0: batch_segment<MCUBES_F_C0, MIXED>(v, sd, cells, hist, seg, it, acc); break;
        case MCUBES_F_DISCONT: batch_segment<MCUBES_F_DISCONT, MIXED>(v, sd, cells, hist, seg, it, acc); break;
        case MCUBES_F_COSMO6: batch_segment<MCUBES_F_COSMO6, MIXED>(v, sd, cells, hist, seg, it, acc); break;
        default: break;
        }
        block_write_sums(acc, red, a.seg_part + 3 * (size_t)si);
        if (seg.adjust) {
            __syncthreads();
            HT* out = reinterpret_cast<HT*>(a.seg_hist) + seg.hist_off;
            for (uint32_t i = threadIdx.x; i < d * nb; i += blockDim.x) out[i] = hist[i];
        }
    }
}

template <bool MIXED>
cudaError_t launch_vsample_batch_prec(const BatchArgs& a, int grid, size_t smem, cudaStream_t s)
{
    auto k = vsample_batch_kernel<MIXED>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kVsThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <bool MIXED>
cudaError_t vsample_batch_occupancy_prec(size_t smem, int* blocks)
{
    auto k = vsample_batch_kernel<MIXED>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, kVsThreads, smem);
}

}  // namespace mc
