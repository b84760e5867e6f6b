// aton_static.cu -- aton_photon_sum_static: the FP64 photon count sum(N) * V of a device
// field, computed without allocating any memory.
//
// Some callers cannot let a library call cudaMalloc: a host code that hands out all device
// memory from its own fixed pool and forbids allocations behind its back, or a monitoring hook
// that runs between time steps, where an allocation could block on work already queued. For
// them this entry point keeps its scratch (one FP64 partial sum per 65536 cells, and the
// result) in a file-scope __device__ array of fixed size, 128 KB plus 256 bytes. Every GPU
// that loads the library holds that array until the process exits.
//
// In host code the array's name is only a host-side stand-in, never a device address: the
// address is looked up once per device with cudaGetSymbolAddress (with that device current)
// on the first call made on that device, and passed to the kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "aton_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kCellsPerPart = kThreads * 256;   // cells summed by one block
constexpr int kMaxParts = 16384;                // scratch partial sums
constexpr long long kMaxCells = (long long)kMaxParts * kCellsPerPart;   // 2^30 = 1024^3
constexpr int kMaxDevices = 64;

// Scratch: kMaxParts partial sums, then the result slot (index kMaxParts).
static __device__ __align__(256) double g_photon_scratch[kMaxParts + 32];

std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Block b sums cells [b * kCellsPerPart, (b + 1) * kCellsPerPart) in FP64, fixed order.
__global__ void __launch_bounds__(kThreads) k_static_partial(const float* N, long long n,
                                                             double* part) {
  __shared__ double s[kThreads];
  const long long base = (long long)blockIdx.x * kCellsPerPart;
  double a = 0.0;
  for (int k = 0; k < kCellsPerPart / kThreads; ++k) {
    const long long i = base + (long long)k * kThreads + threadIdx.x;
    if (i < n) a += (double)N[i];
  }
  s[threadIdx.x] = a;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// One block: the partial sums in a fixed order, times the cell volume, into part[kMaxParts].
__global__ void __launch_bounds__(kThreads) k_static_final(double* part, int nparts, double V) {
  __shared__ double s[kThreads];
  double a = 0.0;
  for (int i = threadIdx.x; i < nparts; i += kThreads) a += part[i];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[kMaxParts] = s[0] * V;
}

int report(int code, const char* msg) {
  aton::set_last_message(msg);
  return code;
}

}  // namespace

extern "C" int aton_photon_sum_static(const float* N, int64_t n, double cell_volume, double* out,
                                      void* stream) {
  char buf[256];
  if (!N || !out) return report(ATON_ERR_BADARG, "N and out must not be NULL");
  if (n < 1) return report(ATON_ERR_BADARG, "n must be >= 1");
  if (n > kMaxCells) {
    snprintf(buf, sizeof(buf),
             "n = %lld exceeds the static scratch limit of %lld cells (%d partial sums)",
             (long long)n, kMaxCells, kMaxParts);
    return report(ATON_ERR_BADARG, buf);
  }
  if (!(cell_volume > 0) || !std::isfinite(cell_volume))
    return report(ATON_ERR_BADARG, "cell_volume must be positive and finite");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return report(ATON_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return report(ATON_ERR_BADARG, "device index out of range");
  cudaPointerAttributes attr;
  e = cudaPointerGetAttributes(&attr, N);
  if (e != cudaSuccess) return report(ATON_ERR_CUDA, cudaGetErrorString(e));
  if ((attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) ||
      attr.device != dev)
    return report(ATON_ERR_BADARG, "N must be device memory of the current device");
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      e = cudaGetSymbolAddress((void**)&g_scratch_addr[dev], g_photon_scratch);
      if (e != cudaSuccess) {
        g_scratch_addr[dev] = nullptr;
        return report(ATON_ERR_CUDA, cudaGetErrorString(e));
      }
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int nparts = (int)((n + kCellsPerPart - 1) / kCellsPerPart);
  k_static_partial<<<nparts, kThreads, 0, s>>>(N, n, scratch);
  k_static_final<<<1, kThreads, 0, s>>>(scratch, nparts, cell_volume);
  e = cudaGetLastError();
  if (e != cudaSuccess) return report(ATON_ERR_CUDA, cudaGetErrorString(e));
  e = cudaMemcpyAsync(out, scratch + kMaxParts, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return report(ATON_ERR_CUDA, cudaGetErrorString(e));
  return ATON_OK;
}
