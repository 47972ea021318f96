// Batched sampling kernel, mixed precision (see batch.cuh).
#include "batch.cuh"

namespace mc {
cudaError_t launch_vsample_batch_mixed(const BatchArgs& a, int grid, size_t smem, cudaStream_t s)
{
    return launch_vsample_batch_prec<true>(a, grid, smem, s);
}
cudaError_t vsample_batch_occupancy_mixed(size_t smem, int* blocks) { return vsample_batch_occupancy_prec<true>(smem, blocks); }
}  // namespace mc
