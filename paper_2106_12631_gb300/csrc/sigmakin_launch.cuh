// Launchers shared by the per-process translation units (one TU per process
// so the four diagram programs compile in parallel).
#pragma once
#include "launch.h"
#include "sigmakin.cuh"
#include "sigmakin_hs.cuh"

namespace mg {

template <class P, class R, int CS>
cudaError_t launch_sigmakin_variant(const SigArgs& a, const Couplings<R>& cp, int64_t grid, cudaStream_t s) {
  using L = SigLayout<P, R, CS>;
  auto k = sigmakin_kernel<P, R, CS>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)grid, SigCfg<P>::NT, L::bytes, s>>>(a, cp);
  return cudaGetLastError();
}

// The helicity-shared kernel runs persistent: as many CTAs as are resident at
// once (SMs x CTAs per SM, cached per device), each looping over groups of
// events (the CTA's group count follows from the mask on the device).  CTAs
// per SM: the larger of the occupancy query and the count the kernel's shared
// memory budget and launch bounds are built for (the query has returned 1 for
// the tcgen05 variant, whose two CTAs per SM fit); should fewer fit, the
// surplus CTAs start later and take their groups then.
// ra != nullptr: the kernel that runs RAMBO itself (sigmakin_hs_rambo_kernel).
template <class P, class R, int CS, bool FUSED = false>
cudaError_t launch_sigmakin_hs_variant(const SigArgs& a, const Couplings<R>& cp, int64_t grid, cudaStream_t s,
                                       const RamboArgs* ra = nullptr) {
  using L = HsLayout<P, R, CS>;
  constexpr int NT = HsCfg<P, R>::NT;
  constexpr int kMaxDevices = 64;
  static int resident[kMaxDevices];  // CTAs resident on the whole device; 0 until known
  const void* k = FUSED ? (const void*)sigmakin_hs_rambo_kernel<P, R, CS> : (const void*)sigmakin_hs_kernel<P, R, CS>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
  if (e != cudaSuccess) return e;
  grid = (a.nevt + HsCfg<P, R>::EVMIN - 1) / HsCfg<P, R>::EVMIN;
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  int cap = dev < kMaxDevices ? resident[dev] : 0;
  if (cap == 0) {
    int nsm = 0, per = 0;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, NT, L::bytes)) != cudaSuccess) return e;
    cap = nsm * (per > HsCfg<P, R>::CTAS ? per : HsCfg<P, R>::CTAS);
    if (dev < kMaxDevices) resident[dev] = cap;
  }
  if (grid > cap) grid = cap;
  if constexpr (FUSED) sigmakin_hs_rambo_kernel<P, R, CS><<<(unsigned)grid, NT, L::bytes, s>>>(a, cp, *ra);
  else sigmakin_hs_kernel<P, R, CS><<<(unsigned)grid, NT, L::bytes, s>>>(a, cp);
  return cudaGetLastError();
}

// mode 0 FP64; 1 mixed, colour sum on CUDA cores below 48 colour flows and on
// the tensor cores from 48 on; 2 mixed + CUDA-core colour sum; 5 mixed +
// tcgen05 colour sum (helicity-shared kernel); 3 FP64, 4 mixed + tcgen05 with
// the per-helicity unrolled kernel (every helicity recomputes all its currents)
inline SigArgs sig_args(const SigLaunch& l) {
  return SigArgs{l.nevt, l.mom, l.mask, l.me, l.mask_out, l.pp, l.hel_rnd, l.hel_out, l.col_rnd, l.col_out};
}

template <class P>
cudaError_t launch_sigmakin_impl(const SigLaunch& l, int mode, cudaStream_t s) {
  const SigArgs a = sig_args(l);
  const int64_t grid = (l.nevt + SigCfg<P>::EVMIN - 1) / SigCfg<P>::EVMIN;
  if (grid == 0) return cudaSuccess;
  constexpr bool tc_default = P::NCOLOR >= 48;
  switch (mode) {
    case 0: return launch_sigmakin_hs_variant<P, double, CS_SIMT>(a, l.cd, grid, s);
    case 1:
      return tc_default ? launch_sigmakin_hs_variant<P, float, CS_TC>(a, l.cf, grid, s)
                        : launch_sigmakin_hs_variant<P, float, CS_SIMT>(a, l.cf, grid, s);
    case 2: return launch_sigmakin_hs_variant<P, float, CS_SIMT>(a, l.cf, grid, s);
    case 5: return launch_sigmakin_hs_variant<P, float, CS_TC>(a, l.cf, grid, s);
    case 3: return launch_sigmakin_variant<P, double, CS_SIMT>(a, l.cd, grid, s);
    case 4: return launch_sigmakin_variant<P, float, CS_TC>(a, l.cf, grid, s);
  }
  return cudaErrorInvalidValue;
}

// RAMBO and SIGMAKIN in one kernel; the helicity-shared modes only (0 FP64,
// 1 mixed, 2 mixed + CUDA-core colour sum, 5 mixed + tcgen05 colour sum)
template <class P>
cudaError_t launch_sigmakin_rambo_impl(const SigLaunch& l, int mode, cudaStream_t s) {
  const SigArgs a = sig_args(l);
  const RamboArgs ra{l.rnd, l.wgt, l.ecm, l.key, l.first_event, l.st};
  if (l.nevt == 0) return cudaSuccess;
  constexpr bool tc_default = P::NCOLOR >= 48;
  switch (mode) {
    case 0: return launch_sigmakin_hs_variant<P, double, CS_SIMT, true>(a, l.cd, 0, s, &ra);
    case 1:
      return tc_default ? launch_sigmakin_hs_variant<P, float, CS_TC, true>(a, l.cf, 0, s, &ra)
                        : launch_sigmakin_hs_variant<P, float, CS_SIMT, true>(a, l.cf, 0, s, &ra);
    case 2: return launch_sigmakin_hs_variant<P, float, CS_SIMT, true>(a, l.cf, 0, s, &ra);
    case 5: return launch_sigmakin_hs_variant<P, float, CS_TC, true>(a, l.cf, 0, s, &ra);
  }
  return cudaErrorInvalidValue;
}

template <class P>
cudaError_t launch_filter_impl(const SigLaunch& l, cudaStream_t s) {
  using L = SigLayout<P, double, CS_SIMT>;
  SigArgs a{l.nevt, l.mom, l.mask, l.me, l.mask_out, l.pp, nullptr, nullptr};
  const int64_t grid = l.nevt * ((P::NHEL + FILTER_NT - 1) / FILTER_NT);
  if (grid == 0) return cudaSuccess;
  auto k = filter_kernel<P>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)grid, FILTER_NT, L::bytes, s>>>(a, l.cd);
  return cudaGetLastError();
}

}  // namespace mg

// The FP64 kernels of a process (sum and filter) are instantiated in their own
// translation unit (MG_INSTANTIATE_FP64), the FP32 ones with the dispatcher.
#define MG_DEFINE_PROCESS_LAUNCHERS(N)                                                                  \
  namespace mg {                                                                                         \
  extern template cudaError_t launch_sigmakin_variant<Proc##N, double, CS_SIMT>(                        \
      const SigArgs&, const Couplings<double>&, int64_t, cudaStream_t);                                  \
  extern template cudaError_t launch_sigmakin_hs_variant<Proc##N, double, CS_SIMT>(                     \
      const SigArgs&, const Couplings<double>&, int64_t, cudaStream_t, const RamboArgs*);                \
  extern template cudaError_t launch_sigmakin_hs_variant<Proc##N, double, CS_SIMT, true>(               \
      const SigArgs&, const Couplings<double>&, int64_t, cudaStream_t, const RamboArgs*);                \
  extern template cudaError_t launch_filter_impl<Proc##N>(const SigLaunch&, cudaStream_t);              \
  cudaError_t launch_sigmakin_p##N(const SigLaunch& a, int mode, cudaStream_t s) {                      \
    return launch_sigmakin_impl<Proc##N>(a, mode, s);                                                    \
  }                                                                                                      \
  cudaError_t launch_sigmakin_rambo_p##N(const SigLaunch& a, int mode, cudaStream_t s) {                \
    return launch_sigmakin_rambo_impl<Proc##N>(a, mode, s);                                              \
  }                                                                                                      \
  cudaError_t launch_filter_p##N(const SigLaunch& a, cudaStream_t s) { return launch_filter_impl<Proc##N>(a, s); } \
  }

#define MG_INSTANTIATE_FP64(N)                                                                          \
  namespace mg {                                                                                         \
  template cudaError_t launch_sigmakin_variant<Proc##N, double, CS_SIMT>(                               \
      const SigArgs&, const Couplings<double>&, int64_t, cudaStream_t);                                  \
  template cudaError_t launch_sigmakin_hs_variant<Proc##N, double, CS_SIMT>(                            \
      const SigArgs&, const Couplings<double>&, int64_t, cudaStream_t, const RamboArgs*);                \
  template cudaError_t launch_sigmakin_hs_variant<Proc##N, double, CS_SIMT, true>(                      \
      const SigArgs&, const Couplings<double>&, int64_t, cudaStream_t, const RamboArgs*);                \
  template cudaError_t launch_filter_impl<Proc##N>(const SigLaunch&, cudaStream_t);                     \
  }
