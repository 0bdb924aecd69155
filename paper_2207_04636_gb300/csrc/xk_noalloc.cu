// Allocation-free exchange-energy reduction.
//
// E_x = -sum_t K[t] C[t] computed like the library's own FP64 reduction, but
// with its partial sums kept in a fixed array of device memory declared in
// this file, so that the call never allocates.  Every process that loads the
// library holds this array (16 KiB) on every device it touches until exit.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "xk_internal.h"

namespace xk {

// Partial sums of one call: one per chunk of kNoAllocChunk elements.
constexpr int kNoAllocParts = 2048;
constexpr int64_t kNoAllocChunk = 2048;
constexpr int64_t kNoAllocMaxCount = (int64_t)kNoAllocParts * kNoAllocChunk;

static __device__ __align__(256) double g_noalloc_parts[kNoAllocParts];

namespace {

constexpr int kTpb = 256;

// Block b sums elements [b*chunk, min(count, (b+1)*chunk)) in a fixed order
// and writes parts[b]; every part the second stage reads is written here.
__global__ void noalloc_stage1(const double* __restrict__ a, const double* __restrict__ b,
                               int64_t count, double* __restrict__ parts) {
  __shared__ double sh[kTpb];
  const int64_t beg = (int64_t)blockIdx.x * kNoAllocChunk;
  const int64_t end = beg + kNoAllocChunk < count ? beg + kNoAllocChunk : count;
  double s = 0.0;
  for (int64_t t = beg + threadIdx.x; t < end; t += kTpb) s = fma(a[t], b[t], s);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kTpb / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) parts[blockIdx.x] = sh[0];
}

__global__ void noalloc_stage2(const double* __restrict__ parts, int nparts, double* out) {
  __shared__ double sh[kTpb];
  double s = 0.0;
  for (int t = threadIdx.x; t < nparts; t += kTpb) s += parts[t];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kTpb / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = -sh[0];
}

// Device address of g_noalloc_parts, resolved once per device.
constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
double* g_addr[kMaxDevices] = {nullptr};

cudaError_t parts_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_parts);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

int64_t noalloc_max_count() { return kNoAllocMaxCount; }

cudaError_t exchange_energy_noalloc(const double* K, const double* C, int64_t count, double* Ex,
                                    cudaStream_t s) {
  double* parts = nullptr;
  cudaError_t e = parts_address(&parts);
  if (e != cudaSuccess) return e;
  const int nparts = count > 0 ? (int)((count + kNoAllocChunk - 1) / kNoAllocChunk) : 1;
  noalloc_stage1<<<nparts, kTpb, 0, s>>>(K, C, count, parts);
  noalloc_stage2<<<1, kTpb, 0, s>>>(parts, nparts, Ex);
  count_launch(2);
  return cudaGetLastError();
}

}  // namespace xk
