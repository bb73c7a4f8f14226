// RAMBO phase-space sampling on the GPU (the paper's toy workflow, Sec. 3:
// random numbers -> RAMBO -> momenta and weights; Kleiss, Stirling and Ellis,
// CPC 40 (1986) 359).  One thread per event, FP64 (kept in FP64 in both
// precision modes), structure-of-arrays loads and stores with the event index
// fastest, so every warp access is one contiguous 256-byte segment.
//
// Per final-state particle i, rows 4i..4i+3 of the random numbers give
//   cos(theta) = 2 r1 - 1, phi = 2 pi r2, q0 = -log(r3 r4);
// the massless momenta q are boosted and scaled to the centre-of-mass frame
// at sqrt(s) = ecm; with masses, a Newton iteration finds the common scale
// xi with sum_i sqrt(m_i^2 + xi^2 E_i^2) = ecm.  Beams are massless along +z
// (leg 0) and -z (leg 1).  The weight is the flat phase-space volume element
// without (2 pi) factors.
#include <cstdint>

#include "launch.h"
#include "rambo.cuh"
#include "rng.cuh"

namespace mg {

// Uniforms of one event: from a buffer rnd[k][nevt], or (rnd == nullptr)
// drawn on the device from the counter-based generator (key, event index).
template <int NF>
__global__ void __launch_bounds__(128) rambo_kernel(int64_t nevt, double ecm, const double* __restrict__ rnd,
                                                    double* __restrict__ mom, double* __restrict__ wgt,
                                                    RamboSetup st, uint64_t key, int64_t first_event) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nevt) return;
  double r[4 * NF];
  if (rnd) {
#pragma unroll
    for (int k = 0; k < 4 * NF; ++k) r[k] = rnd[(int64_t)k * nevt + i];
  } else {
#pragma unroll
    for (int k = 0; k < 4 * NF; ++k) r[k] = sm64_uniform(key, first_event + i, k);
  }
  RamboState<NF> z;
  rambo_forward<NF>(r, ecm, st, z);
  const double h = 0.5 * ecm;
  const int64_t L = 4 * nevt;
  mom[0 * nevt + i] = h; mom[1 * nevt + i] = 0.0; mom[2 * nevt + i] = 0.0; mom[3 * nevt + i] = h;
  mom[L + 0 * nevt + i] = h; mom[L + 1 * nevt + i] = 0.0; mom[L + 2 * nevt + i] = 0.0; mom[L + 3 * nevt + i] = -h;
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) mom[(int64_t)((2 + f) * 4 + mu) * nevt + i] = z.k[f][mu];
  wgt[i] = z.w;
}

// Final-state momenta only, out[4 f + mu][nevt] (the gradient's first pass;
// the beams are fixed), from rnd[k][nevt].
template <int NF>
__global__ void __launch_bounds__(128) rambo_final_kernel(int64_t nevt, double ecm, const double* __restrict__ rnd,
                                                          double* __restrict__ out, RamboSetup st) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nevt) return;
  double r[4 * NF];
#pragma unroll
  for (int k = 0; k < 4 * NF; ++k) r[k] = rnd[(int64_t)k * nevt + i];
  RamboState<NF> z;
  rambo_forward<NF>(r, ecm, st, z);
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) out[(int64_t)(4 * f + mu) * nevt + i] = z.k[f][mu];
}

// RAMBO adjoint: grad[4 f + mu][i] holds dL/dk_f^mu of the final momenta on
// entry; on exit grad[k][i] = dL/d rnd[k][i] (0 for rows RAMBO does not use).
template <int NF>
__global__ void __launch_bounds__(128) rambo_adjoint_kernel(int64_t nevt, double ecm, const double* __restrict__ rnd,
                                                            int nrows, double* __restrict__ grad, RamboSetup st) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nevt) return;
  double r[4 * NF], kb[NF][4], rb[4 * NF];
#pragma unroll
  for (int k = 0; k < 4 * NF; ++k) r[k] = rnd[(int64_t)k * nevt + i];
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) kb[f][mu] = grad[(int64_t)(4 * f + mu) * nevt + i];
  RamboState<NF> z;
  rambo_forward<NF>(r, ecm, st, z);
  rambo_adjoint<NF>(r, ecm, st, z, kb, rb);
  for (int k = 0; k < nrows; ++k) grad[(int64_t)k * nevt + i] = k < 4 * NF ? rb[k] : 0.0;
}

cudaError_t launch_rambo_final(int nfinal, int64_t nevt, double ecm, const double* rnd, double* out,
                               const RamboSetup& st, cudaStream_t s) {
  const int nt = 128;
  const int64_t grid = (nevt + nt - 1) / nt;
  switch (nfinal) {
    case 2: rambo_final_kernel<2><<<(unsigned)grid, nt, 0, s>>>(nevt, ecm, rnd, out, st); break;
    case 3: rambo_final_kernel<3><<<(unsigned)grid, nt, 0, s>>>(nevt, ecm, rnd, out, st); break;
    case 4: rambo_final_kernel<4><<<(unsigned)grid, nt, 0, s>>>(nevt, ecm, rnd, out, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_rambo_adjoint(int nfinal, int64_t nevt, double ecm, const double* rnd, int nrows, double* grad,
                                 const RamboSetup& st, cudaStream_t s) {
  const int nt = 128;
  const int64_t grid = (nevt + nt - 1) / nt;
  switch (nfinal) {
    case 2: rambo_adjoint_kernel<2><<<(unsigned)grid, nt, 0, s>>>(nevt, ecm, rnd, nrows, grad, st); break;
    case 3: rambo_adjoint_kernel<3><<<(unsigned)grid, nt, 0, s>>>(nevt, ecm, rnd, nrows, grad, st); break;
    case 4: rambo_adjoint_kernel<4><<<(unsigned)grid, nt, 0, s>>>(nevt, ecm, rnd, nrows, grad, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_rambo(int nfinal, int64_t nevt, double ecm, const double* rnd, double* mom, double* wgt,
                         const RamboSetup& st, cudaStream_t s, uint64_t seed, int64_t first_event) {
  const int nt = 128;
  const int64_t grid = (nevt + nt - 1) / nt;
  const uint64_t key = sm64_mix(seed);
  switch (nfinal) {
    case 2: rambo_kernel<2><<<(unsigned)grid, nt, 0, s>>>(nevt, ecm, rnd, mom, wgt, st, key, first_event); break;
    case 3: rambo_kernel<3><<<(unsigned)grid, nt, 0, s>>>(nevt, ecm, rnd, mom, wgt, st, key, first_event); break;
    case 4: rambo_kernel<4><<<(unsigned)grid, nt, 0, s>>>(nevt, ecm, rnd, mom, wgt, st, key, first_event); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace mg
