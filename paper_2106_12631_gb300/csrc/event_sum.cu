// Event accumulation in FP64 (the paper's validation and cross-section
// estimate, Sec. 3: the average matrix element over all events of a run):
// out = (sum w_i me_i, sum (w_i me_i)^2, N), by a two-pass tree reduction
// whose order depends only on N, so repeated runs agree bit for bit.
//
// Pass 1: block b sums events [b*CHUNK, (b+1)*CHUNK) -> partial[b] (2 doubles)
// in caller-provided scratch; pass 2: one block reduces the partials.
#include <cstdint>
#include <mutex>

#include "launch.h"

namespace mg {

constexpr int kSumThreads = 256;
constexpr int kSumItems = 16;
constexpr int64_t kSumChunk = (int64_t)kSumThreads * kSumItems;

__device__ __forceinline__ void block_tree_sum(double* s1, double* s2) {
  for (int off = kSumThreads / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) {
      s1[threadIdx.x] += s1[threadIdx.x + off];
      s2[threadIdx.x] += s2[threadIdx.x + off];
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kSumThreads) event_sum_pass1(int64_t n, const double* __restrict__ me,
                                                                const double* __restrict__ w,
                                                                double* __restrict__ partial) {
  __shared__ double s1[kSumThreads], s2[kSumThreads];
  const int64_t base = (int64_t)blockIdx.x * kSumChunk;
  double a = 0.0, b = 0.0;
#pragma unroll
  for (int k = 0; k < kSumItems; ++k) {
    const int64_t i = base + (int64_t)k * kSumThreads + threadIdx.x;
    if (i < n) {
      const double x = me[i] * w[i];
      a += x;
      b += x * x;
    }
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  block_tree_sum(s1, s2);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = s1[0];
    partial[2 * blockIdx.x + 1] = s2[0];
  }
}

__global__ void __launch_bounds__(kSumThreads) event_sum_pass2(int64_t nblk, const double* __restrict__ partial,
                                                                double* __restrict__ out3, int64_t n) {
  __shared__ double s1[kSumThreads], s2[kSumThreads];
  double a = 0.0, b = 0.0;
  for (int64_t k = threadIdx.x; k < nblk; k += kSumThreads) {
    a += partial[2 * k];
    b += partial[2 * k + 1];
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  block_tree_sum(s1, s2);
  if (threadIdx.x == 0) {
    out3[0] = s1[0];
    out3[1] = s2[0];
    out3[2] = (double)n;
  }
}

int64_t event_sum_blocks(int64_t n) { return n > 0 ? (n + kSumChunk - 1) / kSumChunk : 0; }

cudaError_t launch_event_sum(int64_t n, const double* me, const double* w, double* out3, double* partial,
                             cudaStream_t s) {
  const int64_t nblk = event_sum_blocks(n);
  if (nblk > 0) event_sum_pass1<<<(unsigned)nblk, kSumThreads, 0, s>>>(n, me, w, partial);
  event_sum_pass2<<<1, kSumThreads, 0, s>>>(nblk, partial, out3, n);
  return cudaGetLastError();
}

// ---- allocation-free variant --------------------------------------------
// Partials live in a fixed device array instead of caller scratch, for callers
// that cannot allocate device memory.  One array per loaded library on every
// device, shared by all calls; pass 1 writes every partial pass 2 reads, so no
// clearing is needed, but calls that overlap on the GPU (e.g. on two streams)
// race on it.
constexpr int64_t kNoAllocMaxEvents = int64_t(1) << 26;
constexpr int64_t kNoAllocMaxBlocks = kNoAllocMaxEvents / kSumChunk;
static __device__ __align__(256) double g_noalloc_partials[2 * kNoAllocMaxBlocks];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {};
}  // namespace

int64_t event_sum_noalloc_max_events() { return kNoAllocMaxEvents; }

// Device address of the array on the current device, looked up once per
// device (the host-side symbol is only a stand-in and must not be passed to a
// kernel).
cudaError_t event_sum_noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

cudaError_t launch_event_sum_noalloc(int64_t n, const double* me, const double* w, double* out3, cudaStream_t s) {
  double* partial = nullptr;
  cudaError_t e = event_sum_noalloc_scratch(&partial);
  if (e != cudaSuccess) return e;
  const int64_t nblk = event_sum_blocks(n);
  if (nblk > 0) event_sum_pass1<<<(unsigned)nblk, kSumThreads, 0, s>>>(n, me, w, partial);
  event_sum_pass2<<<1, kSumThreads, 0, s>>>(nblk, partial, out3, n);
  return cudaGetLastError();
}

}  // namespace mg
