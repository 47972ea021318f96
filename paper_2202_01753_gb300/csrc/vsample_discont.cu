// Sampling kernels for the discont integrand family (see vsample.cuh).
#include "vsample.cuh"

MC_INSTANTIATE_FAMILY(MCUBES_F_DISCONT, discont)
