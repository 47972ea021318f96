// Sampling kernels for the prodpeak integrand family (see vsample.cuh).
#include "vsample.cuh"

MC_INSTANTIATE_FAMILY(MCUBES_F_PRODPEAK, prodpeak)
