// Batched sampling kernels for the c0 integrand family (see batch.cuh).
#include "batch.cuh"

MC_INSTANTIATE_BATCH_FAMILY(MCUBES_F_C0, c0)
