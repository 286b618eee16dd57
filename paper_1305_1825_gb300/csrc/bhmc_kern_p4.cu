// Kernels of the treecode Monte Carlo instantiated for multipole order p = 4.
#define BHMC_P 4
#include "bhmc_kernels_impl.cuh"
