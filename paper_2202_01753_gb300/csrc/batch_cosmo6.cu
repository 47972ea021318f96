// Batched sampling kernels for the cosmo6 integrand family (see batch.cuh).
#include "batch.cuh"

MC_INSTANTIATE_BATCH_FAMILY(MCUBES_F_COSMO6, cosmo6)
