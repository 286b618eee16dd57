// bhmc_noalloc.cu -- direct-sum total energy without any device allocation.
//
// bhmc_energy_direct() obtains its per-block partial sums from cudaMalloc.
// Some callers cannot allocate device memory at the moment they need the
// energy: code that runs while a CUDA stream is being captured into a graph
// (allocation calls are illegal there), host functions enqueued with
// cudaLaunchHostFunc (they may not call the CUDA API at all, and allocation
// also synchronises the device), and host applications that own the whole
// device-memory budget and hand this library only pre-allocated buffers.
// This file gives them a variant of the same FP64 O(N^2) kernel whose scratch
// is a fixed array in the library's own device image.
#include <mutex>

#include "../../include/bhmc.h"
#include "bhmc_common.cuh"

namespace {

constexpr int kBlock = 256;
constexpr int kMaxBlocks = 4096;  // one partial sum per block
constexpr int kMaxDevices = 64;

// File-scope scratch: every device that loads the library holds these 32 KiB
// until the process exits.  Calls share it; each call writes exactly the
// partials it reads back, so nothing has to be cleared between calls, but two
// calls whose kernels overlap on one device race on it.
static __device__ __align__(256) double g_partials[kMaxBlocks];

// Device address of g_partials per device.  In host code the symbol is only a
// host-side stand-in, so the address is looked up once per device, with that
// device current.
double* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

__global__ void __launch_bounds__(kBlock) k_pair_rows(const double* q, const double* xyz, int n,
                                                      double* partial) {
  __shared__ double red[kBlock / 32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (i < n) {
    const double xi = xyz[3 * i], yi = xyz[3 * i + 1], zi = xyz[3 * i + 2];
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      const double dx = xyz[3 * j] - xi, dy = xyz[3 * j + 1] - yi, dz = xyz[3 * j + 2] - zi;
      s += q[j] / sqrt(dx * dx + dy * dy + dz * dz);
    }
    acc = q[i] * s;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) t += red[w];
    partial[blockIdx.x] = t;
  }
}

__global__ void k_sum_partials(const double* partial, int nblk, double half_lB, double* E) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int k = threadIdx.x; k < nblk; k += blockDim.x) acc += partial[k];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *E = half_lB * t;
  }
}

}  // namespace

extern "C" bhmc_status bhmc_energy_direct_noalloc(int64_t n, const double* q, const double* xyz, double lB,
                                                  double* E, void* cuda_stream) {
  if (n < 1 || !q || !xyz || !E) return BHMC_EINVAL;
  if (n > (int64_t)kMaxBlocks * kBlock) return BHMC_ESCRATCH;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BHMC_ECUDA;
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) return BHMC_ECUDA;
      g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int nblk = (int)((n + kBlock - 1) / kBlock);
  k_pair_rows<<<nblk, kBlock, 0, st>>>(q, xyz, (int)n, scratch);
  k_sum_partials<<<1, 1024, 0, st>>>(scratch, nblk, 0.5 * lB, E);
  return cudaGetLastError() == cudaSuccess ? BHMC_OK : BHMC_ECUDA;
}
