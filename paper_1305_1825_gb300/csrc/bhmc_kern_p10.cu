// Kernels of the treecode Monte Carlo instantiated for multipole order p = 10.
#define BHMC_P 10
#include "bhmc_kernels_impl.cuh"
