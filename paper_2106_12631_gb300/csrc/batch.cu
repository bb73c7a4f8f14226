// Momenta of an external integrator, one event after another ([nevt][npar][4],
// array of structures), into the kernels' structure of arrays ([npar][4][nevt],
// event index fastest), through a shared-memory tile of 32 events so that both
// the loads and the stores are coalesced.
#include <cstdint>

#include "launch.h"

namespace mg {

constexpr int kAosEvents = 32;
constexpr int kAosThreads = 256;
constexpr int kAosMaxComp = 4 * 8;

__global__ void __launch_bounds__(kAosThreads) aos_to_soa_kernel(int64_t nevt, int ncomp, const double* __restrict__ aos,
                                                                double* __restrict__ soa) {
  __shared__ double tile[kAosEvents][kAosMaxComp + 1];
  const int64_t e0 = (int64_t)blockIdx.x * kAosEvents;
  const int nloc = (int)((nevt - e0) < kAosEvents ? (nevt - e0) : kAosEvents);
  for (int t = threadIdx.x; t < nloc * ncomp; t += kAosThreads) tile[t / ncomp][t % ncomp] = aos[e0 * ncomp + t];
  __syncthreads();
  for (int t = threadIdx.x; t < ncomp * kAosEvents; t += kAosThreads) {
    const int c = t / kAosEvents, e = t % kAosEvents;
    if (e < nloc) soa[(int64_t)c * nevt + e0 + e] = tile[e][c];
  }
}

cudaError_t launch_aos_to_soa(int64_t nevt, int npar, const double* aos, double* soa, cudaStream_t s) {
  if (4 * npar > kAosMaxComp) return cudaErrorInvalidValue;
  const int64_t grid = (nevt + kAosEvents - 1) / kAosEvents;
  aos_to_soa_kernel<<<(unsigned)grid, kAosThreads, 0, s>>>(nevt, 4 * npar, aos, soa);
  return cudaGetLastError();
}

}  // namespace mg
