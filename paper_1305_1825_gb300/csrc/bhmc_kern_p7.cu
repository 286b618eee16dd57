// Kernels of the treecode Monte Carlo instantiated for multipole order p = 7.
#define BHMC_P 7
#include "bhmc_kernels_impl.cuh"
