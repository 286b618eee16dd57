// Kernels of the treecode Monte Carlo instantiated for multipole order p = 3.
#define BHMC_P 3
#include "bhmc_kernels_impl.cuh"
