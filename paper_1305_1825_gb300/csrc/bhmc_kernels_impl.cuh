// bhmc_kernels_impl.cuh -- definitions of the per-order launchers; included by
// one translation unit per multipole order with BHMC_P defined.
#pragma once

#include "bhmc_launch.cuh"
#include "bhmc_move.cuh"
#include "bhmc_energy.cuh"
#include "bhmc_forces.cuh"

namespace bhmc {


template <>
cudaError_t launch_delta<BHMC_P>(const SysDev& S, int warps, int i, const double* b, DeltaOut* out,
                                 cudaStream_t st) {
  if (S.prec == BHMC_PREC_F64)
    k_delta<BHMC_P, double, BHMC_LAYOUT_SOA><<<1, 32 * warps, 0, st>>>(S, i, b[0], b[1], b[2], out);
  else if (S.layout == BHMC_LAYOUT_AOS)
    k_delta<BHMC_P, float, BHMC_LAYOUT_AOS><<<1, 32 * warps, 0, st>>>(S, i, b[0], b[1], b[2], out);
  else
    k_delta<BHMC_P, float, BHMC_LAYOUT_SOA><<<1, 32 * warps, 0, st>>>(S, i, b[0], b[1], b[2], out);
  return cudaGetLastError();
}

template <>
cudaError_t launch_step<BHMC_P>(const SysDev& S, int warps, unsigned long long m, unsigned replica,
                                unsigned long long seed, double step, MoveRec* rec,
                                bhmc_mc_stats* stats, cudaStream_t st) {
  const uint2 key = make_uint2((unsigned)seed, (unsigned)(seed >> 32));
  if (S.prec == BHMC_PREC_F64)
    k_step<BHMC_P, double, BHMC_LAYOUT_SOA><<<1, 32 * warps, 0, st>>>(S, m, replica, key, step, rec, stats);
  else if (S.layout == BHMC_LAYOUT_AOS)
    k_step<BHMC_P, float, BHMC_LAYOUT_AOS><<<1, 32 * warps, 0, st>>>(S, m, replica, key, step, rec, stats);
  else
    k_step<BHMC_P, float, BHMC_LAYOUT_SOA><<<1, 32 * warps, 0, st>>>(S, m, replica, key, step, rec, stats);
  return cudaGetLastError();
}

template <>
cudaError_t launch_step_mala<BHMC_P>(const SysDev& S, int warps, unsigned long long m, unsigned replica,
                                     unsigned long long seed, double tau, MoveRec* rec, bhmc_mc_stats* stats,
                                     cudaStream_t st) {
  const uint2 key = make_uint2((unsigned)seed, (unsigned)(seed >> 32));
  if (S.prec == BHMC_PREC_F64)
    k_step_mala<BHMC_P, double, BHMC_LAYOUT_SOA><<<1, 32 * warps, 0, st>>>(S, m, replica, key, tau, rec, stats);
  else if (S.layout == BHMC_LAYOUT_AOS)
    k_step_mala<BHMC_P, float, BHMC_LAYOUT_AOS><<<1, 32 * warps, 0, st>>>(S, m, replica, key, tau, rec, stats);
  else
    k_step_mala<BHMC_P, float, BHMC_LAYOUT_SOA><<<1, 32 * warps, 0, st>>>(S, m, replica, key, tau, rec, stats);
  return cudaGetLastError();
}

template <typename Kern>
static cudaError_t launch_cluster(Kern kern, int proposals, int warps, cudaStream_t st, const SysDev& S,
                                  unsigned long long move0, unsigned long long n, uint2 key, double step,
                                  MoveRec* rec, bhmc_mc_stats* stats) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)proposals, 1, 1);
  cfg.blockDim = dim3((unsigned)(32 * warps), 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)proposals;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, S, move0, n, 0u, key, step, rec, stats);
}

template <>
cudaError_t launch_spec<BHMC_P>(const SysDev& S, int warps, int proposals, unsigned long long move0,
                                unsigned long long n_moves, unsigned long long seed, double step, MoveRec* rec,
                                bhmc_mc_stats* stats, cudaStream_t st) {
  const uint2 key = make_uint2((unsigned)seed, (unsigned)(seed >> 32));
  if (S.prec == BHMC_PREC_F64)
    return launch_cluster(k_spec<BHMC_P, double, BHMC_LAYOUT_SOA>, proposals, warps, st, S, move0, n_moves, key,
                          step, rec, stats);
  if (S.layout == BHMC_LAYOUT_AOS)
    return launch_cluster(k_spec<BHMC_P, float, BHMC_LAYOUT_AOS>, proposals, warps, st, S, move0, n_moves, key,
                          step, rec, stats);
  return launch_cluster(k_spec<BHMC_P, float, BHMC_LAYOUT_SOA>, proposals, warps, st, S, move0, n_moves, key, step,
                        rec, stats);
}

template <typename Kern>
static cudaError_t launch_cluster_batch(Kern kern, int proposals, int warps, int n_rep, cudaStream_t st,
                                        const SysDev* views, const BatchArgs* args, bhmc_mc_stats* stats) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(proposals * n_rep), 1, 1);
  cfg.blockDim = dim3((unsigned)(32 * warps), 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)proposals;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, views, n_rep, args, stats);
}

template <>
cudaError_t launch_spec_batch<BHMC_P>(const SysDev& S0, int warps, int proposals, const SysDev* views, int n_rep,
                                      const BatchArgs* args, bhmc_mc_stats* stats, cudaStream_t st) {
  if (S0.prec == BHMC_PREC_F64)
    return launch_cluster_batch(k_spec_batch<BHMC_P, double, BHMC_LAYOUT_SOA>, proposals, warps, n_rep, st, views,
                                args, stats);
  if (S0.layout == BHMC_LAYOUT_AOS)
    return launch_cluster_batch(k_spec_batch<BHMC_P, float, BHMC_LAYOUT_AOS>, proposals, warps, n_rep, st, views,
                                args, stats);
  return launch_cluster_batch(k_spec_batch<BHMC_P, float, BHMC_LAYOUT_SOA>, proposals, warps, n_rep, st, views,
                              args, stats);
}

template <>
cudaError_t launch_batch<BHMC_P>(const SysDev& S0, int warps, const SysDev* views, int n_rep, int grid,
                                 const BatchArgs* args, bhmc_mc_stats* stats, cudaStream_t st) {
  if (S0.prec == BHMC_PREC_F64)
    k_batch<BHMC_P, double, BHMC_LAYOUT_SOA><<<grid, 32 * warps, 0, st>>>(views, n_rep, args, stats);
  else if (S0.layout == BHMC_LAYOUT_AOS)
    k_batch<BHMC_P, float, BHMC_LAYOUT_AOS><<<grid, 32 * warps, 0, st>>>(views, n_rep, args, stats);
  else
    k_batch<BHMC_P, float, BHMC_LAYOUT_SOA><<<grid, 32 * warps, 0, st>>>(views, n_rep, args, stats);
  return cudaGetLastError();
}

template <>
int batch_occupancy<BHMC_P>(const SysDev& S0, int warps) {
  int n = 0;
  if (S0.prec == BHMC_PREC_F64)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<BHMC_P, double, BHMC_LAYOUT_SOA>, 32 * warps, 0);
  else if (S0.layout == BHMC_LAYOUT_AOS)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<BHMC_P, float, BHMC_LAYOUT_AOS>, 32 * warps, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<BHMC_P, float, BHMC_LAYOUT_SOA>, 32 * warps, 0);
  return n;
}

template <>
cudaError_t launch_energy<BHMC_P>(const SysDev& S, int warps, int grid, double* partial, double* phi,
                                  int* err, unsigned long long* cnt, cudaStream_t st) {
  if (S.prec == BHMC_PREC_F64)
    k_energy<BHMC_P, double, BHMC_LAYOUT_SOA><<<grid, 32 * warps, 0, st>>>(S, S.order, partial, phi, err, cnt);
  else if (S.layout == BHMC_LAYOUT_AOS)
    k_energy<BHMC_P, float, BHMC_LAYOUT_AOS><<<grid, 32 * warps, 0, st>>>(S, S.order, partial, phi, err, cnt);
  else
    k_energy<BHMC_P, float, BHMC_LAYOUT_SOA><<<grid, 32 * warps, 0, st>>>(S, S.order, partial, phi, err, cnt);
  return cudaGetLastError();
}

template <>
cudaError_t launch_forces<BHMC_P>(const SysDev& S, int grid, double* phi, double* tgrad, double* lam,
                                  double* psi, double* src, int* err, cudaStream_t st) {
  if (S.prec == BHMC_PREC_F64)
    k_forces_traverse<BHMC_P, double, BHMC_LAYOUT_SOA><<<grid, 128, 0, st>>>(S, S.order, phi, tgrad, lam, psi, src, err);
  else if (S.layout == BHMC_LAYOUT_AOS)
    k_forces_traverse<BHMC_P, float, BHMC_LAYOUT_AOS><<<grid, 128, 0, st>>>(S, S.order, phi, tgrad, lam, psi, src, err);
  else
    k_forces_traverse<BHMC_P, float, BHMC_LAYOUT_SOA><<<grid, 128, 0, st>>>(S, S.order, phi, tgrad, lam, psi, src, err);
  return cudaGetLastError();
}

}  // namespace bhmc
