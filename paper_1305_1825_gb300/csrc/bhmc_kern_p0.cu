// Kernels of the treecode Monte Carlo instantiated for multipole order p = 0.
#define BHMC_P 0
#include "bhmc_kernels_impl.cuh"
