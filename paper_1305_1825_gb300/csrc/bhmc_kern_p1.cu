// Kernels of the treecode Monte Carlo instantiated for multipole order p = 1.
#define BHMC_P 1
#include "bhmc_kernels_impl.cuh"
