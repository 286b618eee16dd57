// Kernels of the treecode Monte Carlo instantiated for multipole order p = 2.
#define BHMC_P 2
#include "bhmc_kernels_impl.cuh"
