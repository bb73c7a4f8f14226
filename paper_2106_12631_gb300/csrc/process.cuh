// The four processes: generated diagram programs plus the per-process
// constants the kernels need.
#pragma once
#include "helas_adj.cuh"

// CTA barrier inside the straight-line contraction code every MG_HS_LOCK_EVERY
// amplitudes (at the next change of amputated current), so that the warps
// stay close together in the program and share instruction fetches (0: none)
#ifndef MG_HS_LOCK_EVERY
#define MG_HS_LOCK_EVERY 0
#endif
#define HS_LOCKSTEP(m, n)                                                             \
  do {                                                                                \
    constexpr int lock_every_ = MG_HS_LOCK_EVERY > 0 ? MG_HS_LOCK_EVERY : 1 << 30;    \
    if constexpr ((m) / lock_every_ != (n) / lock_every_) __syncthreads();            \
  } while (0)
#include "gen/proc1.cuh"
#include "gen/proc2.cuh"
#include "gen/proc3.cuh"
#include "gen/proc4.cuh"

namespace mg {

// Propagator factor of one internal line, formed in FP64 from the FP64
// outgoing momentum sum K:  fermion (top)  i / (K^2 - mt^2 + i mt wt),
// vector -i / (K^2 - M^2 + i M W)  with M = 0 for gluon and photon, M = mZ for
// the Z.  The denominator is the only place near a pole (Z, top) where
// cancellation in K^2 - M^2 matters; both precision modes form it in FP64.
__device__ __forceinline__ void propagator_fp64(const double* K, int kind, const PhysParams& pp,
                                                double& re, double& im) {
  const double k2 = K[0] * K[0] - K[1] * K[1] - K[2] * K[2] - K[3] * K[3];
  double dr = k2, di = 0.0;
  if (kind == 1) { dr = k2 - pp.mt * pp.mt; di = pp.mt * pp.wt; }
  else if (kind == 3) { dr = k2 - pp.mz * pp.mz; di = pp.mz * pp.wz; }
  // 1/(dr + i di) = (dr - i di)/|d|^2 ; fermion: times i, vector: times -i
  const double inv = 1.0 / (dr * dr + di * di);
  const double ar = dr * inv, ai = -di * inv;
  if (kind == 1) { re = -ai; im = ar; }
  else { re = ai; im = -ar; }
}

}  // namespace mg
