// Sampling kernels for the interpolation-table integrand family (see vsample.cuh).
#include "vsample.cuh"

MC_INSTANTIATE_FAMILY(MCUBES_F_TABLE, table)
