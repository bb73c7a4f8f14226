// Launchers shared by the per-process translation units (one TU per process
// so the four diagram programs compile in parallel).
#pragma once
#include "launch.h"
#include "sigmakin.cuh"

namespace mg {

template <class P>
cudaError_t launch_sigmakin_impl(const SigLaunch& l, int mode, cudaStream_t s) {
  SigArgs a{l.nevt, l.mom, l.mask, l.me, l.mask_out, l.pp};
  const int64_t grid = (l.nevt + SigCfg<P>::EVMIN - 1) / SigCfg<P>::EVMIN;
  if (grid == 0) return cudaSuccess;
  switch (mode) {
    case 0: sigmakin_kernel<P, double><<<(unsigned)grid, kSigmaThreads, 0, s>>>(a, l.cd); break;
    case 1:
    case 2: sigmakin_kernel<P, float><<<(unsigned)grid, kSigmaThreads, 0, s>>>(a, l.cf); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class P>
cudaError_t launch_filter_impl(const SigLaunch& l, cudaStream_t s) {
  SigArgs a{l.nevt, l.mom, l.mask, l.me, l.mask_out, l.pp};
  const int64_t grid = (l.nevt + SigCfg<P>::EVMIN - 1) / SigCfg<P>::EVMIN;
  if (grid == 0) return cudaSuccess;
  filter_kernel<P><<<(unsigned)grid, kSigmaThreads, 0, s>>>(a, l.cd);
  return cudaGetLastError();
}

}  // namespace mg

#define MG_DEFINE_PROCESS_LAUNCHERS(N)                                                              \
  namespace mg {                                                                                     \
  cudaError_t launch_sigmakin_p##N(const SigLaunch& a, int mode, cudaStream_t s) {                  \
    return launch_sigmakin_impl<Proc##N>(a, mode, s);                                                \
  }                                                                                                  \
  cudaError_t launch_filter_p##N(const SigLaunch& a, cudaStream_t s) { return launch_filter_impl<Proc##N>(a, s); } \
  }
