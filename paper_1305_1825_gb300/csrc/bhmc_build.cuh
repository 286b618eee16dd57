// bhmc_build.cuh -- launchers of the build, stand-alone commit and direct-sum kernels.
#pragma once

#include "bhmc_common.cuh"

namespace bhmc {

cudaError_t build_init_charges(const SysDev& S, const double* q, const double* xyz, int* flags,
                               cudaStream_t st);
cudaError_t build_keys(const SysDev& S, int* perm, int* flags, cudaStream_t st);
cudaError_t build_root(const SysDev& S, int* seg, cudaStream_t st);
cudaError_t build_split_level(const SysDev& S, const int* list, int n_list, int base_group, int depth,
                              int* perm, int* perm2, int* seg, int* next_flags, cudaStream_t st);
cudaError_t build_compact(const int* in, int n, int* out, int* n_out, cudaStream_t st);
cudaError_t build_leaves_moments(const SysDev& S, int n_nodes, const int* perm, const int* seg, int* flags,
                                 const int* level_begin, int n_levels, cudaStream_t st);
// Evaluation coefficients W32 of every cluster in use from the FP64 moments.
cudaError_t launch_wmirror(const SysDev& S, cudaStream_t st);
// Sets flags[1] when two mobile ions of the built tree overlap (hard cores).
cudaError_t launch_hard_core_check(const SysDev& S, int* flags, cudaStream_t st);
// Adds the radial counts and charges of the mobile ions to counts[nbins], charge[nbins] (device).
cudaError_t launch_radial_counts(const SysDev& S, int nbins, double lo, double hi, double width,
                                 unsigned long long* counts, double* charge, cudaStream_t st);
cudaError_t launch_commit(const SysDev& S, int i, const double* b, int* status, cudaStream_t st);
cudaError_t launch_direct_energy(const SysDev& S, double* partial, int nblk, cudaStream_t st);
cudaError_t launch_interleave(const SysDev& S, double* q, double* xyz, cudaStream_t st);
// fixed charges held outside the tree (fixed_direct): every pair with a fixed
// charge, exactly.  Energy pass: each fixed charge's potential (phi[f], may be
// null, zeroed by the caller; qphi[f] = q_f phi_f for f < n_fix) and the
// fixed charges' potential at every tree charge (added to phi[j];
// qphi[n_fix] += sum_j q_j phi_fixed(r_j)); qphi zeroed by the caller.  Force
// pass: the same pairs' target and source terms added to the adjoint arrays.
cudaError_t launch_fixed_targets(const SysDev& S, double* phi, double* qphi, cudaStream_t st);
cudaError_t launch_forces_fixed(const SysDev& S, double* phi, double* tgrad, double* psi, double* src,
                                cudaStream_t st);

}  // namespace bhmc
