// Sampling kernels for the cosmo6 integrand family (see vsample.cuh).
#include "vsample.cuh"

MC_INSTANTIATE_FAMILY(MCUBES_F_COSMO6, cosmo6)
