// Cross section and hit-or-miss unweighting on the device — the last steps of
// the toy workflow (Sec. 3): the weighted events x_i = w_i |M_i|^2 estimate the
// cross section, and unweighting keeps event i with probability x_i / max x,
// so that the kept events are distributed as |M|^2 over phase space.
//
// Unweighting is deterministic: the uniform of event i comes from the
// counter-based generator (seed, first_event + i, row 63); event i is kept
// iff u_i * max x < x_i (so x_i <= 0 is never kept); the kept indices are
// written in increasing order (stable compaction from a block scan).
// Launches: per-block maxima, their maximum, per-block counts, an exclusive
// scan of the counts (also the total), and the scatter of the indices.
#include <cstdint>

#include "launch.h"
#include "rng.cuh"

namespace mg {

constexpr int kUwThreads = 256;
constexpr int kUwPerThread = 4;
constexpr int kUwBlock = kUwThreads * kUwPerThread;  // events per block
constexpr int kUwScanThreads = 1024;

int64_t unweight_blocks(int64_t n) { return (n + kUwBlock - 1) / kUwBlock; }

__device__ __forceinline__ double uw_x(const double* __restrict__ me, const double* __restrict__ w, int64_t i) {
  return w[i] * me[i];
}

// block maximum of x over the block's events (-inf when it has none)
__global__ void __launch_bounds__(kUwThreads) uw_max_blocks(int64_t n, const double* __restrict__ me,
                                                            const double* __restrict__ w, double* part) {
  __shared__ double red[kUwThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kUwBlock + (int64_t)threadIdx.x * kUwPerThread;
  double m = -INFINITY;
#pragma unroll
  for (int j = 0; j < kUwPerThread; ++j)
    if (base + j < n) m = fmax(m, uw_x(me, w, base + j));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < kUwThreads / 32 ? red[threadIdx.x] : -INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) part[blockIdx.x] = m;
  }
}

// maximum of the block maxima (one CTA)
__global__ void __launch_bounds__(kUwScanThreads) uw_max_final(int64_t nblk, const double* part, double* xmax) {
  __shared__ double red[kUwScanThreads / 32];
  double m = -INFINITY;
  for (int64_t b = threadIdx.x; b < nblk; b += kUwScanThreads) m = fmax(m, part[b]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = red[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) *xmax = m;
  }
}

// kept events among a thread's kUwPerThread consecutive events, as a bit mask
__device__ __forceinline__ unsigned uw_keep(int64_t n, const double* __restrict__ me, const double* __restrict__ w,
                                            uint64_t key, int64_t first_event, double xmax, int64_t base) {
  unsigned bits = 0;
#pragma unroll
  for (int j = 0; j < kUwPerThread; ++j) {
    const int64_t i = base + j;
    if (i < n && sm64_uniform(key, first_event + i, kRngRowUnweight) * xmax < uw_x(me, w, i)) bits |= 1u << j;
  }
  return bits;
}

// exclusive prefix sum of v over the CTA (kUwThreads threads); total in *tot
__device__ __forceinline__ int uw_block_scan(int v, int* tot) {
  __shared__ int wsum[kUwThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int s = lane < kUwThreads / 32 ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kUwThreads / 32) wsum[lane] = s;  // inclusive warp totals
  }
  __syncthreads();
  const int before = (warp > 0 ? wsum[warp - 1] : 0) + x - v;
  *tot = wsum[kUwThreads / 32 - 1];
  return before;
}

__global__ void __launch_bounds__(kUwThreads) uw_count_blocks(int64_t n, const double* __restrict__ me,
                                                              const double* __restrict__ w, uint64_t key,
                                                              int64_t first_event, const double* xmax,
                                                              int64_t* counts) {
  const int64_t base = (int64_t)blockIdx.x * kUwBlock + (int64_t)threadIdx.x * kUwPerThread;
  const int c = __popc(uw_keep(n, me, w, key, first_event, *xmax, base));
  int tot;
  uw_block_scan(c, &tot);
  if (threadIdx.x == 0) counts[blockIdx.x] = tot;
}

// exclusive scan of the block counts in place (one CTA); the total into *count
__global__ void __launch_bounds__(kUwScanThreads) uw_scan_counts(int64_t nblk, int64_t* counts, int64_t* count) {
  __shared__ int64_t part[kUwScanThreads];
  const int64_t per = (nblk + kUwScanThreads - 1) / kUwScanThreads;
  const int64_t b0 = threadIdx.x * per, b1 = b0 + per < nblk ? b0 + per : nblk;
  int64_t s = 0;
  for (int64_t b = b0; b < b1; ++b) s += counts[b];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {  // fixed-order scan of kUwScanThreads partial sums
    int64_t acc = 0;
    for (int t = 0; t < kUwScanThreads; ++t) {
      const int64_t v = part[t];
      part[t] = acc;
      acc += v;
    }
    *count = acc;
  }
  __syncthreads();
  int64_t acc = part[threadIdx.x];
  for (int64_t b = b0; b < b1; ++b) {
    const int64_t v = counts[b];
    counts[b] = acc;
    acc += v;
  }
}

__global__ void __launch_bounds__(kUwThreads) uw_write(int64_t n, const double* __restrict__ me,
                                                       const double* __restrict__ w, uint64_t key,
                                                       int64_t first_event, const double* xmax,
                                                       const int64_t* offsets, int64_t* idx) {
  const int64_t base = (int64_t)blockIdx.x * kUwBlock + (int64_t)threadIdx.x * kUwPerThread;
  const unsigned bits = uw_keep(n, me, w, key, first_event, *xmax, base);
  int tot;
  int64_t pos = offsets[blockIdx.x] + uw_block_scan(__popc(bits), &tot);
#pragma unroll
  for (int j = 0; j < kUwPerThread; ++j)
    if (bits >> j & 1u) idx[pos++] = base + j;
}

cudaError_t launch_unweight(int64_t n, const double* me, const double* w, uint64_t seed, int64_t first_event,
                            int64_t* idx, int64_t* count, double* scratch, cudaStream_t s) {
  const int64_t nblk = unweight_blocks(n);
  double* xmax = scratch;
  double* part = scratch + 1;
  int64_t* counts = reinterpret_cast<int64_t*>(scratch + 1 + nblk);
  const uint64_t key = sm64_mix(seed);
  uw_max_blocks<<<(unsigned)nblk, kUwThreads, 0, s>>>(n, me, w, part);
  uw_max_final<<<1, kUwScanThreads, 0, s>>>(nblk, part, xmax);
  uw_count_blocks<<<(unsigned)nblk, kUwThreads, 0, s>>>(n, me, w, key, first_event, xmax, counts);
  uw_scan_counts<<<1, kUwScanThreads, 0, s>>>(nblk, counts, count);
  uw_write<<<(unsigned)nblk, kUwThreads, 0, s>>>(n, me, w, key, first_event, xmax, counts, idx);
  return cudaGetLastError();
}

// sigma = norm * mean(x), error = norm * sqrt(sample variance / N), from the
// event sums {sum x, sum x^2, N}
__global__ void xsec_kernel(const double* sums, double norm, double* out) {
  const double n = sums[2];
  const double mean = n > 0 ? sums[0] / n : 0.0;
  const double var = n > 1 ? (sums[1] / n - mean * mean) * (n / (n - 1)) : 0.0;
  out[0] = norm * mean;
  out[1] = n > 0 ? norm * sqrt(fmax(var, 0.0) / n) : 0.0;
}

cudaError_t launch_cross_section(const double* sums, double norm, double* out, cudaStream_t s) {
  xsec_kernel<<<1, 1, 0, s>>>(sums, norm, out);
  return cudaGetLastError();
}

}  // namespace mg
