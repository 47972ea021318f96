// Batched sampling kernels for the discont integrand family (see batch.cuh).
#include "batch.cuh"

MC_INSTANTIATE_BATCH_FAMILY(MCUBES_F_DISCONT, discont)
