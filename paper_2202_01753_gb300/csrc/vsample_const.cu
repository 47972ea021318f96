// Sampling kernels for the const integrand family (see vsample.cuh).
#include "vsample.cuh"

MC_INSTANTIATE_FAMILY(MCUBES_F_CONST, const)
