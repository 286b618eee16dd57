// bhmc_taylor.cuh -- Taylor coefficients T_n of 1/|r| (Sec. 3.1 recurrence) and
// the p-th order particle-cluster approximation of Eq. (3.3), fully unrolled so
// that every coefficient lives in a register.
#pragma once

#include "bhmc_common.cuh"

namespace bhmc {

template <typename R>
__device__ __forceinline__ R rsqrt_t(R v);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float v) {
  return rsqrtf(v);
}
template <>
__device__ __forceinline__ double rsqrt_t<double>(double v) {
  return 1.0 / sqrt(v);
}

// T_n(R) for ||n|| <= P in graded order:
//   T_0 = 1/r,  T_n = -[(2k-1)/k sum_i R_i T_{n-e_i} + (k-1)/k sum_i T_{n-2e_i}] / r^2,
// k = ||n||, the recurrence of Sec. 3.1 divided by k r^2.
template <int P, typename R>
__device__ __forceinline__ void taylor(R x, R y, R z, R (&T)[nterms(P)]) {
  const R r2 = x * x + y * y + z * z;
  const R rinv = rsqrt_t<R>(r2);
  const R ir2 = rinv * rinv;
  T[0] = rinv;
#pragma unroll
  for (int k = 1; k <= P; ++k) {
    const R a = R(2 * k - 1) / R(k);
    const R b = R(k - 1) / R(k);
#pragma unroll
    for (int n1 = k; n1 >= 0; --n1) {
#pragma unroll
      for (int n2 = k - n1; n2 >= 0; --n2) {
        const int n3 = k - n1 - n2;
        R s1 = R(0), s2 = R(0);
        if (n1 >= 1) s1 += x * T[tidx(n1 - 1, n2, n3)];
        if (n2 >= 1) s1 += y * T[tidx(n1, n2 - 1, n3)];
        if (n3 >= 1) s1 += z * T[tidx(n1, n2, n3 - 1)];
        if (k >= 2) {
          if (n1 >= 2) s2 += T[tidx(n1 - 2, n2, n3)];
          if (n2 >= 2) s2 += T[tidx(n1, n2 - 2, n3)];
          if (n3 >= 2) s2 += T[tidx(n1, n2, n3 - 2)];
        }
        T[tidx(n1, n2, n3)] = -(a * s1 + b * s2) * ir2;
      }
    }
  }
}

}  // namespace bhmc
