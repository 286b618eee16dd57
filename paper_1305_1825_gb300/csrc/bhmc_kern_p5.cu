// Kernels of the treecode Monte Carlo instantiated for multipole order p = 5.
#define BHMC_P 5
#include "bhmc_kernels_impl.cuh"
