// Batched sampling kernels for the prodpeak integrand family (see batch.cuh).
#include "batch.cuh"

MC_INSTANTIATE_BATCH_FAMILY(MCUBES_F_PRODPEAK, prodpeak)
