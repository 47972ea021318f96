// Sampling kernels for the gauss integrand family (see vsample.cuh).
#include "vsample.cuh"

MC_INSTANTIATE_FAMILY(MCUBES_F_GAUSS, gauss)
