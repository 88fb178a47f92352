// Lagrangian reduction E = sum tbar * Omega without any device allocation
// and without a caller-provided workspace.
//
// Who needs this: callers that cannot allocate device memory at the point
// where they want E -- for example a solver loop whose device memory is
// owned by another framework's pool (so it has no way to hand us a
// workspace), or code that must not pay the implicit device
// synchronisation of cudaMalloc/cudaFree inside its iteration.  They pass
// only the inputs (tbar2 and Omega, device buffers they already own) and
// the output E; the partial sums of the reduction live in a fixed device
// array that belongs to this file.
//
// The scratch array below is part of the library image: every GPU that
// loads the library holds it (kNoAllocMaxSys * kNoAllocBlocks doubles,
// 512 KiB) until the process exits.  All calls share it and it keeps the
// last call's contents; each call overwrites exactly the entries it later
// reads, so nothing needs clearing, but calls that overlap on the GPU
// (different streams, or different host threads on one device) race on it.
#include <mutex>

#include "ccladder.h"
#include "gemm.h"

namespace ccl {
namespace {

constexpr int kNoAllocMaxSys = 64;    // systems per call (the size limit)
constexpr int kNoAllocBlocks = 1024;  // partial sums per system
constexpr int kNoAllocThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxSys * kNoAllocBlocks];

// Host-side addresses of g_noalloc_partials, one per device, resolved on the
// first call made with that device current.
std::mutex g_na_mu;
double* g_na_ptr[kMaxDevices] = {nullptr};

__device__ __forceinline__ double block_sum_na(double x) {
  __shared__ double red[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = x;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  x = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (w == 0) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
  }
  return x;
}

// Block b of system s writes part[s * kNoAllocBlocks + b] (all of them).
__global__ void k_noalloc_dot(const double* __restrict__ x, const double* __restrict__ y, long long n,
                              double* __restrict__ part) {
  double acc = 0.0;
  for (long long k = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; k < n;
       k += static_cast<long long>(gridDim.x) * blockDim.x)
    acc += x[k] * y[k];
  acc = block_sum_na(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_noalloc_final(const double* __restrict__ part, double* __restrict__ out) {
  double acc = 0.0;
  for (int k = threadIdx.x; k < kNoAllocBlocks; k += blockDim.x) acc += part[k];
  acc = block_sum_na(acc);
  if (threadIdx.x == 0) *out = acc;
}

int scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CC_ERR_DEVICE;
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess || !p) {
      note_cuda(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
      return CC_ERR_CUDA;
    }
    g_na_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_na_ptr[dev];
  return CC_OK;
}

}  // namespace
}  // namespace ccl

using namespace ccl;

extern "C" int cc_ladder_lagrangian_noalloc(const cc_ladder_system* sys, int n_sys, double* E,
                                            double* const* omega, void* stream) {
  if (!sys || n_sys < 1 || !E || !omega) return CC_ERR_ARG;
  if (n_sys > kNoAllocMaxSys) return CC_ERR_SIZE;
  if (reinterpret_cast<uintptr_t>(E) & 7) return CC_ERR_ARG;
  for (int i = 0; i < n_sys; ++i) {
    const cc_ladder_system& s = sys[i];
    if (s.o < 1 || s.v < 1 || !s.tbar2 || !omega[i]) return CC_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(s.tbar2) | reinterpret_cast<uintptr_t>(omega[i])) & 7) return CC_ERR_ARG;
  }
  int dev = 0, maj = 0, mnr = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&mnr, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess || maj != 10 || mnr != 3)
    return CC_ERR_DEVICE;
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < n_sys; ++i) {
    const long long n = static_cast<long long>(sys[i].o) * sys[i].o * sys[i].v * sys[i].v;
    double* part = scratch + static_cast<long long>(i) * kNoAllocBlocks;
    k_noalloc_dot<<<kNoAllocBlocks, kNoAllocThreads, 0, st>>>(sys[i].tbar2, omega[i], n, part);
    k_noalloc_final<<<1, kNoAllocThreads, 0, st>>>(part, E + i);
    count_launch(2);
  }
  const cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    note_cuda(e);
    return CC_ERR_CUDA;
  }
  return CC_OK;
}
