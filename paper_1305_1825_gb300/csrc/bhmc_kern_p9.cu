// Kernels of the treecode Monte Carlo instantiated for multipole order p = 9.
#define BHMC_P 9
#include "bhmc_kernels_impl.cuh"
