// rks_sketch_apply_noalloc: z = Omega x without any allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's device-memory pool (the pool already owns the memory, so a
// private allocation can fail or fragment it) and latency-critical loops that
// cannot afford the device-wide synchronisation that cudaFree implies.  For
// them this entry point keeps its scratch (the FP64 sketch sums and a status
// word) in a fixed file-scope device array instead of allocating it.
//
// The array is a host-side symbol: host code must not pass its name to a
// kernel.  On the first call on each device (with that device current) the
// device address is resolved once with cudaGetSymbolAddress and cached for
// the process (a cudaDeviceReset invalidates it).

#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/rks.h"
#include "rks_impl.h"

// d sums, then the status word in the tail (one double wide).  Every GPU that
// loads the library holds one copy (64 KB + 8 B) until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[RKS_NOALLOC_MAX_D + 1];

namespace {

constexpr int kMaxDevices = 64;

std::mutex g_mu;
double* g_addr[kMaxDevices] = {nullptr};

__global__ void k_noalloc_scale(int d, double scale, const double* __restrict__ sums, double* __restrict__ z) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < d; r += gridDim.x * blockDim.x) z[r] = sums[r] * scale;
}

// Device address of the scratch on the current device (resolved once).
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RKS_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return RKS_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return RKS_ECUDA;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return RKS_OK;
}

}  // namespace

extern "C" int rks_sketch_apply_noalloc(int64_t n, int d, int zeta, uint64_t seed, const double* x, double* z,
                                        void* stream) {
  if (n <= 0 || zeta < 1 || zeta > 16 || d < 2 * zeta || d > RKS_NOALLOC_MAX_D || !x || !z) return RKS_EINVAL;
  double* sums = nullptr;
  int rc = scratch_address(&sums);
  if (rc) return rc;
  if (rks::configure_kernels() != cudaSuccess) return RKS_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  int* flag = reinterpret_cast<int*>(sums + RKS_NOALLOC_MAX_D);
  // the array keeps the previous call's contents: clear what must start at zero
  if (cudaMemsetAsync(sums, 0, (size_t)d * sizeof(double), st) != cudaSuccess ||
      cudaMemsetAsync(flag, 0, sizeof(int), st) != cudaSuccess)
    return RKS_ECUDA;
  rks::launch_sketch_vec(n, x, 1.0, d, zeta, seed, sums, flag, st);
  k_noalloc_scale<<<(d + 255) / 256, 256, 0, st>>>(d, 1.0 / std::sqrt((double)zeta), sums, z);
  if (cudaGetLastError() != cudaSuccess) return RKS_ECUDA;
  int f = 0;
  if (cudaMemcpyAsync(&f, flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return RKS_ECUDA;
  return f ? RKS_EINVAL : RKS_OK;
}
