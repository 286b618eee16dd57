// bhmc_noalloc.cu -- direct-sum total energy without any device allocation.
//
// bhmc_energy_direct() obtains its per-block partial sums from cudaMalloc.
// Some callers cannot call cudaMalloc when they need the energy: applications
// that reserve the device memory they will use up front and give libraries
// only pre-allocated buffers (a later allocation would fail, or break their
// memory accounting), and loops that must not take the implicit device-wide
// synchronisation a cudaMalloc/cudaFree pair can cause.  This file gives them
// a variant of the same FP64 O(N^2) kernel whose scratch is a fixed array in
// the library's own device image.
#include <cuda.h>

#include <mutex>

#include "../../include/bhmc.h"
#include "bhmc_common.cuh"

namespace {

constexpr int kBlock = 256;
constexpr int kMaxBlocks = 4096;  // one partial sum per block
constexpr int kMaxContexts = 64;

// File-scope scratch: every device that loads the library holds these 32 KiB
// until the process exits.  Calls share it; each call writes exactly the
// partials it reads back, so nothing has to be cleared between calls, but two
// calls whose kernels overlap on one device race on it.
static __device__ __align__(256) double g_partials[kMaxBlocks];

// In host code g_partials names only a host-side stand-in, so its device
// address is looked up with the context current.  The address belongs to that
// context: it is cached under the context's unique id, which a device reset or
// another context on the same device does not share, so neither can reuse a
// stale address.
struct ScratchEntry {
  unsigned long long ctx_id;
  double* ptr;
};
ScratchEntry g_scratch[kMaxContexts] = {};
int g_n_scratch = 0;
int g_evict = 0;  // next entry to recycle once the table is full (oldest first)
std::mutex g_scratch_mutex;

using PfnCtxGetCurrent = CUresult (*)(CUcontext*);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long*);

// Id of the calling thread's current context (the runtime makes the device's
// primary context current if there is none).  Driver entry points come through
// the runtime, so the library needs no link against the driver library.
bool current_context_id(unsigned long long* id) {
  static PfnCtxGetCurrent get_current = nullptr;
  static PfnCtxGetId get_id = nullptr;
  if (!get_current || !get_id) {
    void* f0 = nullptr;
    void* f1 = nullptr;
    cudaDriverEntryPointQueryResult q0, q1;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess || !f0 || !f1)
      return false;
    get_current = reinterpret_cast<PfnCtxGetCurrent>(f0);
    get_id = reinterpret_cast<PfnCtxGetId>(f1);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS) return false;
  if (!ctx) {
    // no context yet on this thread: cudaSetDevice makes the device's primary
    // context current (it allocates nothing)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess) return false;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
  }
  return get_id(ctx, id) == CUDA_SUCCESS;
}

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
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    unsigned long long id = 0;
    if (!current_context_id(&id)) return BHMC_ECUDA;
    for (int k = 0; k < g_n_scratch; ++k)
      if (g_scratch[k].ctx_id == id) scratch = g_scratch[k].ptr;
    if (!scratch) {
      // first call in this context: look the scratch's device address up
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) return BHMC_ECUDA;
      scratch = static_cast<double*>(p);
      // a full table recycles its oldest entry
      int slot;
      if (g_n_scratch < kMaxContexts) {
        slot = g_n_scratch++;
      } else {
        slot = g_evict;
        g_evict = (g_evict + 1) % kMaxContexts;
      }
      g_scratch[slot].ctx_id = id;
      g_scratch[slot].ptr = scratch;
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int nblk = (int)((n + kBlock - 1) / kBlock);
  k_pair_rows<<<nblk, kBlock, 0, st>>>(q, xyz, (int)n, scratch);
  k_sum_partials<<<1, 1024, 0, st>>>(scratch, nblk, 0.5 * lB, E);
  return cudaGetLastError() == cudaSuccess ? BHMC_OK : BHMC_ECUDA;
}
