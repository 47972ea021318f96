// Sampling kernels for the c0 integrand family (see vsample.cuh).
#include "vsample.cuh"

MC_INSTANTIATE_FAMILY(MCUBES_F_C0, c0)
