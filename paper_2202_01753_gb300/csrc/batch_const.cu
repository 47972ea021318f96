// Batched sampling kernels for the const integrand family (see batch.cuh).
#include "batch.cuh"

MC_INSTANTIATE_BATCH_FAMILY(MCUBES_F_CONST, const)
