// Batched sampling kernel, double precision (see batch.cuh).
#include "batch.cuh"

namespace mc {
cudaError_t launch_vsample_batch_fp64(const BatchArgs& a, int grid, size_t smem, cudaStream_t s)
{
    return launch_vsample_batch_prec<false>(a, grid, smem, s);
}
cudaError_t vsample_batch_occupancy_fp64(size_t smem, int* blocks) { return vsample_batch_occupancy_prec<false>(smem, blocks); }
}  // namespace mc
