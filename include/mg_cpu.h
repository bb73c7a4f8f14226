/* SIMD CPU build of the helicity-shared matrix-element program (the paper's
 * C++ vectorised build, Sec. 4: the same event-parallel code compiled for the
 * host cores, several events per SIMD vector).  A CPU baseline beside the
 * GPU kernels, not a fallback for them: nothing in libmg.so calls it.
 *
 * Built by the package's build step as libmg_cpu.so with the host compiler
 * (portable vector extensions, no target-specific flags: 128-bit NEON on the
 * Grace host, SSE2 on x86-64).  All buffers are HOST memory. */
#ifndef MG_CPU_H
#define MG_CPU_H
#include <stdint.h>

#include "mg.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Events per SIMD vector for a precision (0 FP64, 1 FP32 amplitudes with
 * FP64 momentum sums, propagator denominators and helicity sum). */
int mgc_lanes(int precision);

/* |M|^2 per event, as mg_sigmakin (Sec. 2 and 4: wavefunctions, currents,
 * amplitudes into colour flows, colour sum, helicity sum over mask[h] != 0):
 * mom [npar][4][nevt] host FP64 in the layout of mg_rambo, mask [nhel] host
 * int32, params (the values mg_get_params returns, say), me [nevt] host
 * FP64 out.
 * nthreads >= 1 host threads over blocks of mgc_lanes events.  Returns
 * MG_OK, MG_ERR_PROC or MG_ERR_ARG. */
int mgc_sigmakin(int proc, int64_t nevt, const double* mom, const int32_t* mask, int precision,
                 const mg_params* params, double* me, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
