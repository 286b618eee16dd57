// bhmc_launch.cuh -- host launchers of the kernels that are instantiated per
// multipole order p (one translation unit per p so they compile in parallel).
#pragma once

#include "bhmc_common.cuh"

namespace bhmc {

struct DeltaOut;
struct MoveRec;

template <int P>
cudaError_t launch_delta(const SysDev& S, int warps, int i, const double* b, DeltaOut* out,
                         cudaStream_t st);
template <int P>
cudaError_t launch_step(const SysDev& S, int warps, unsigned long long m, unsigned replica,
                        unsigned long long seed, double step, MoveRec* rec, bhmc_mc_stats* stats,
                        cudaStream_t st);
template <int P>
cudaError_t launch_step_mala(const SysDev& S, int warps, unsigned long long m, unsigned replica,
                             unsigned long long seed, double tau, MoveRec* rec, bhmc_mc_stats* stats,
                             cudaStream_t st);
template <int P>
cudaError_t launch_spec(const SysDev& S, int warps, int proposals, unsigned long long move0,
                        unsigned long long n_moves, unsigned long long seed, double step, MoveRec* rec,
                        bhmc_mc_stats* stats, cudaStream_t st);
template <int P>
cudaError_t launch_spec_batch(const SysDev& S0, int warps, int proposals, const SysDev* views, int n_rep,
                              const BatchArgs* args, bhmc_mc_stats* stats, cudaStream_t st);
template <int P>
cudaError_t launch_batch(const SysDev& S0, int warps, const SysDev* views, int n_rep, int grid,
                         const BatchArgs* args, bhmc_mc_stats* stats, cudaStream_t st);
template <int P>
int batch_occupancy(const SysDev& S0, int warps);
template <int P>
cudaError_t launch_energy(const SysDev& S, int warps, int grid, double* partial, double* phi, int* err,
                          unsigned long long* cnt,
                          cudaStream_t st);

template <int P>
cudaError_t launch_forces(const SysDev& S, int grid, double* phi, double* tgrad, double* lam, double* psi,
                          double* src, int* err, cudaStream_t st);
cudaError_t launch_forces_push(const SysDev& S, const double* phi, const double* tgrad, const double* lam,
                               const double* psi, const double* src, double* dEdr, double* dEdq,
                               cudaStream_t st);

#define BHMC_EXTERN_P(P)                                                                         \
  template <> cudaError_t launch_delta<P>(const SysDev&, int, int, const double*, DeltaOut*, \
                                              cudaStream_t);                                     \
  template <> cudaError_t launch_step<P>(const SysDev&, int, unsigned long long, unsigned,   \
                                             unsigned long long, double, MoveRec*,               \
                                             bhmc_mc_stats*, cudaStream_t);                      \
  template <> cudaError_t launch_step_mala<P>(const SysDev&, int, unsigned long long, unsigned,              \
                                              unsigned long long, double, MoveRec*, bhmc_mc_stats*,        \
                                              cudaStream_t);                                               \
  template <> cudaError_t launch_spec<P>(const SysDev&, int, int, unsigned long long,         \
                                        unsigned long long, unsigned long long, double, MoveRec*,  \
                                        bhmc_mc_stats*, cudaStream_t);                             \
  template <> cudaError_t launch_spec_batch<P>(const SysDev&, int, int, const SysDev*, int,   \
                                              const BatchArgs*, bhmc_mc_stats*, cudaStream_t);  \
  template <> cudaError_t launch_batch<P>(const SysDev&, int, const SysDev*, int, int,       \
                                              const BatchArgs*, bhmc_mc_stats*,                  \
                                              cudaStream_t);                                     \
  template <> int batch_occupancy<P>(const SysDev&, int);                                    \
  template <> cudaError_t launch_energy<P>(const SysDev&, int, int, double*, double*, int*, unsigned long long*, \
                                           cudaStream_t);                                                  \
  template <> cudaError_t launch_forces<P>(const SysDev&, int, double*, double*, double*, double*, double*, int*, \
                                           cudaStream_t);

BHMC_EXTERN_P(0)
BHMC_EXTERN_P(1)
BHMC_EXTERN_P(2)
BHMC_EXTERN_P(3)
BHMC_EXTERN_P(4)
BHMC_EXTERN_P(5)
BHMC_EXTERN_P(6)
BHMC_EXTERN_P(7)
BHMC_EXTERN_P(8)
BHMC_EXTERN_P(9)
BHMC_EXTERN_P(10)

}  // namespace bhmc
