// Internal launch interface between the C ABI (mg_api.cu) and the kernel
// translation units.  Not part of the public header.
#pragma once
#include <cstdint>
#include <functional>
#include <cuda_runtime.h>

#include "mg_types.cuh"
#include "rambo.cuh"

namespace mg {


struct SigLaunch {
  int64_t nevt;
  const double* mom;
  const int32_t* mask;
  double* me;
  int32_t* mask_out;
  PhysParams pp;
  Couplings<double> cd;
  Couplings<float> cf;
  const double* hel_rnd = nullptr;  // helicity and colour-flow choices (helicity-shared kernel only)
  int32_t* hel_out = nullptr;
  const double* col_rnd = nullptr;
  int32_t* col_out = nullptr;
  // RAMBO inside SIGMAKIN (mg_sigmakin_rambo, mg_sigmakin_seeded)
  const double* rnd = nullptr;  // [nrows][nevt], or nullptr: uniforms from (key, first_event + i, row)
  double* wgt = nullptr;
  double ecm = 0.0;
  uint64_t key = 0;
  int64_t first_event = 0;
  RamboSetup st{};
};

// rnd == nullptr: uniforms drawn on the device from (seed, first_event + i, row)
cudaError_t launch_rambo(int nfinal, int64_t nevt, double ecm, const double* rnd, double* mom, double* wgt,
                         const RamboSetup& st, cudaStream_t s, uint64_t seed = 0, int64_t first_event = 0);
// gradient passes: final momenta out[4 f + mu][nevt]; adjoint from grad rows
// 0 .. 4 nfinal - 1 (dL/dk) to dL/d rnd in place
cudaError_t launch_rambo_final(int nfinal, int64_t nevt, double ecm, const double* rnd, double* out,
                               const RamboSetup& st, cudaStream_t s);
cudaError_t launch_rambo_adjoint(int nfinal, int64_t nevt, double ecm, const double* rnd, int nrows, double* grad,
                                 const RamboSetup& st, cudaStream_t s);
// [nevt][npar][4] -> [npar][4][nevt]
cudaError_t launch_aos_to_soa(int64_t nevt, int npar, const double* aos, double* soa, cudaStream_t s);
int64_t unweight_blocks(int64_t n);
cudaError_t launch_unweight(int64_t n, const double* me, const double* w, uint64_t seed, int64_t first_event,
                            int64_t* idx, int64_t* count, double* scratch, cudaStream_t s);
cudaError_t launch_cross_section(const double* sums, double norm, double* out, cudaStream_t s);
int64_t event_sum_blocks(int64_t n);
cudaError_t launch_event_sum(int64_t n, const double* me, const double* w, double* out3, double* partial,
                             cudaStream_t s);
int64_t event_sum_noalloc_max_events();
cudaError_t launch_event_sum_noalloc(int64_t n, const double* me, const double* w, double* out3, cudaStream_t s);

// Kernel-split variant (sigmakin_split.cuh): the launches of one batch, chunk
// by chunk, captured into a CUDA graph and replayed while the key (launch
// arguments and buffers) is unchanged.
struct SplitOps {
  std::function<cudaError_t()> prepare;  // function attributes, before any capture
  std::function<cudaError_t(int64_t first, int64_t last, void* rec, cudaStream_t)> currents;
  std::function<cudaError_t(int64_t first, int64_t last, const void* rec, cudaStream_t)> amplitudes;
};
cudaError_t run_split_graph(const void* key, size_t key_bytes, int64_t nevt, int64_t chunk, void* buf0, void* buf1,
                            const SplitOps& ops, cudaStream_t s);
// per process: record bytes per event (mode 0 FP64, 2 mixed) and the launch
int64_t split_record_bytes_p1(int mode);
int64_t split_record_bytes_p2(int mode);
int64_t split_record_bytes_p3(int mode);
int64_t split_record_bytes_p4(int mode);
cudaError_t launch_sigmakin_split_p1(const SigLaunch& a, int mode, void* ws, int64_t ws_bytes, cudaStream_t s);
cudaError_t launch_sigmakin_split_p2(const SigLaunch& a, int mode, void* ws, int64_t ws_bytes, cudaStream_t s);
cudaError_t launch_sigmakin_split_p3(const SigLaunch& a, int mode, void* ws, int64_t ws_bytes, cudaStream_t s);
cudaError_t launch_sigmakin_split_p4(const SigLaunch& a, int mode, void* ws, int64_t ws_bytes, cudaStream_t s);

// mode: 0 FP64, 1 mixed (tensor-core colour sum), 2 mixed (CUDA-core colour sum)
cudaError_t launch_sigmakin_p1(const SigLaunch& a, int mode, cudaStream_t s);
cudaError_t launch_sigmakin_p2(const SigLaunch& a, int mode, cudaStream_t s);
cudaError_t launch_sigmakin_p3(const SigLaunch& a, int mode, cudaStream_t s);
cudaError_t launch_sigmakin_p4(const SigLaunch& a, int mode, cudaStream_t s);
// RAMBO + SIGMAKIN in one kernel (helicity-shared modes 0, 1, 2, 5 only)
cudaError_t launch_sigmakin_rambo_p1(const SigLaunch& a, int mode, cudaStream_t s);
cudaError_t launch_sigmakin_rambo_p2(const SigLaunch& a, int mode, cudaStream_t s);
cudaError_t launch_sigmakin_rambo_p3(const SigLaunch& a, int mode, cudaStream_t s);
cudaError_t launch_sigmakin_rambo_p4(const SigLaunch& a, int mode, cudaStream_t s);
struct GradLaunch {
  int64_t nevt;
  double ecm;
  const double* rnd;
  int nrows;
  const int32_t* mask;
  const double* gout;  // dL/dme per event, or null for 1
  double* grad;        // [nrows][nevt]
  double* me;          // [nevt] or null
  PhysParams pp;
  Couplings<double> cd;
  Couplings<float> cf;
  RamboSetup st;
};
// mode 0: FP64 forward and adjoint; 1, 2: FP32 forward and adjoint (FP64 RAMBO,
// denominators and sums)
cudaError_t launch_grad_p2(const GradLaunch& a, int mode, cudaStream_t s);
cudaError_t launch_grad_p3(const GradLaunch& a, int mode, cudaStream_t s);

cudaError_t launch_filter_p1(const SigLaunch& a, cudaStream_t s);
cudaError_t launch_filter_p2(const SigLaunch& a, cudaStream_t s);
cudaError_t launch_filter_p3(const SigLaunch& a, cudaStream_t s);
cudaError_t launch_filter_p4(const SigLaunch& a, cudaStream_t s);

}  // namespace mg
