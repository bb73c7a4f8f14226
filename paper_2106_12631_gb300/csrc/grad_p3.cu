// Adjoint gradient d me / d rnd for process 3 (see grad_hs.cuh, grad.cuh, gen/proc3.cuh).
#include "grad_hs.cuh"
#include "launch.h"
namespace mg {
cudaError_t launch_grad_p3(const GradLaunch& a, int mode, cudaStream_t s) { return launch_grad_impl<Proc3>(a, mode, s); }
}  // namespace mg
