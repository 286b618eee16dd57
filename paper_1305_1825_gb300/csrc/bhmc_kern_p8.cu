// Kernels of the treecode Monte Carlo instantiated for multipole order p = 8.
#define BHMC_P 8
#include "bhmc_kernels_impl.cuh"
