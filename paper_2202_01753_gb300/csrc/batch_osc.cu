// Batched sampling kernels for the osc integrand family (see batch.cuh).
#include "batch.cuh"

MC_INSTANTIATE_BATCH_FAMILY(MCUBES_F_OSC, osc)
