"""Parity bars shared by the GPU tests (the CUDA path against the FP64 oracle).

* dE and potentials with the FP32 traversal:
      |x_gpu - x_oracle| <= REL |x_oracle| + FLOOR32 * A,
  A = l_B sum over the interaction lists of |term| (the oracle's abs_sum).  A
  pure relative bar is unattainable as x -> 0: the terms cancel while each FP32
  term (float-pair difference, r^2, rsqrt, charge and weight products) keeps a
  relative error of a few 2^-24.  Their worst-case sum is about 8 * 2^-24 * A =
  4.8e-7 A, but the per-term errors are independent roundings and add like a
  random walk; the measured maximum over the parity suite is about 5e-8 A, so
  the bar is 1e-7 A.
* FP64 traversal: |x_gpu - x_oracle| <= FLOOR64 * A (summation order only).
"""
REL = 1e-5
FLOOR32 = 1e-7
FLOOR64 = 1e-12
