// Sampling kernels for the corner integrand family (see vsample.cuh).
#include "vsample.cuh"

MC_INSTANTIATE_FAMILY(MCUBES_F_CORNER, corner)
