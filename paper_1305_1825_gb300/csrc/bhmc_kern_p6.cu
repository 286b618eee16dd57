// Kernels of the treecode Monte Carlo instantiated for multipole order p = 6.
#define BHMC_P 6
#include "bhmc_kernels_impl.cuh"
