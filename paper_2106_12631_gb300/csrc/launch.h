// Internal launch interface between the C ABI (mg_api.cu) and the kernel
// translation units.  Not part of the public header.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "mg_types.cuh"

namespace mg {

struct RamboSetup {
  double w0;       // flat massless volume (pi/2)^(n-1) s^(n-2) / ((n-1)! (n-2)!)
  int massive;     // any final-state mass != 0
  double xi0;      // Newton start sqrt(1 - (sum m / ecm)^2)
  double m2[4];    // final-state masses squared
};

struct SigLaunch {
  int64_t nevt;
  const double* mom;
  const int32_t* mask;
  double* me;
  int32_t* mask_out;
  PhysParams pp;
  Couplings<double> cd;
  Couplings<float> cf;
};

cudaError_t launch_rambo(int nfinal, int64_t nevt, double ecm, const double* rnd, double* mom, double* wgt,
                         const RamboSetup& st, cudaStream_t s);
int64_t event_sum_blocks(int64_t n);
cudaError_t launch_event_sum(int64_t n, const double* me, const double* w, double* out3, double* partial,
                             cudaStream_t s);
int64_t event_sum_noalloc_max_events();
cudaError_t launch_event_sum_noalloc(int64_t n, const double* me, const double* w, double* out3, cudaStream_t s);

// mode: 0 FP64, 1 mixed (tensor-core colour sum), 2 mixed (CUDA-core colour sum)
cudaError_t launch_sigmakin_p1(const SigLaunch& a, int mode, cudaStream_t s);
cudaError_t launch_sigmakin_p2(const SigLaunch& a, int mode, cudaStream_t s);
cudaError_t launch_sigmakin_p3(const SigLaunch& a, int mode, cudaStream_t s);
cudaError_t launch_sigmakin_p4(const SigLaunch& a, int mode, cudaStream_t s);
cudaError_t launch_filter_p1(const SigLaunch& a, cudaStream_t s);
cudaError_t launch_filter_p2(const SigLaunch& a, cudaStream_t s);
cudaError_t launch_filter_p3(const SigLaunch& a, cudaStream_t s);
cudaError_t launch_filter_p4(const SigLaunch& a, cudaStream_t s);

}  // namespace mg
