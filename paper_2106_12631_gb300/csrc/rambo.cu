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

namespace mg {

template <int NF>
__global__ void __launch_bounds__(128) rambo_kernel(int64_t nevt, double ecm, const double* __restrict__ rnd,
                                                    double* __restrict__ mom, double* __restrict__ wgt,
                                                    RamboSetup st) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nevt) return;
  double q[NF][4];
  double Q[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const double r1 = rnd[(int64_t)(4 * f + 0) * nevt + i];
    const double r2 = rnd[(int64_t)(4 * f + 1) * nevt + i];
    const double r3 = rnd[(int64_t)(4 * f + 2) * nevt + i];
    const double r4 = rnd[(int64_t)(4 * f + 3) * nevt + i];
    const double c = 2.0 * r1 - 1.0;
    const double s = sqrt(1.0 - c * c);
    const double phi = 6.283185307179586477 * r2;
    double sp, cp;
    sincos(phi, &sp, &cp);
    const double e = -log(r3 * r4);
    q[f][0] = e; q[f][1] = e * s * cp; q[f][2] = e * s * sp; q[f][3] = e * c;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) Q[mu] += q[f][mu];
  }
  const double M = sqrt(Q[0] * Q[0] - Q[1] * Q[1] - Q[2] * Q[2] - Q[3] * Q[3]);
  const double b[3] = {-Q[1] / M, -Q[2] / M, -Q[3] / M};
  const double g = Q[0] / M;
  const double a = 1.0 / (1.0 + g);
  const double x = ecm / M;
  double p[NF][4];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const double bq = b[0] * q[f][1] + b[1] * q[f][2] + b[2] * q[f][3];
    p[f][0] = x * (g * q[f][0] + bq);
#pragma unroll
    for (int k = 0; k < 3; ++k) p[f][k + 1] = x * (q[f][k + 1] + b[k] * q[f][0] + a * bq * b[k]);
  }
  double w = st.w0;
  if (st.massive) {
    double xi = st.xi0;
    int extra = 0;
    for (int it = 0; it < 50; ++it) {
      double fv = -ecm, df = 0.0;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const double e = sqrt(st.m2[f] + xi * xi * p[f][0] * p[f][0]);
        fv += e;
        df += xi * p[f][0] * p[f][0] / e;
      }
      xi -= fv / df;
      if (fabs(fv) <= 1e-15 * ecm && ++extra >= 2) break;
    }
    double w2 = 1.0, w3 = 0.0;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const double kk = xi * p[f][0];
      const double e = sqrt(st.m2[f] + kk * kk);
#pragma unroll
      for (int k = 1; k < 4; ++k) p[f][k] *= xi;
      p[f][0] = e;
      w2 *= kk / e;
      w3 += kk * kk / e;
    }
    double pw = 1.0;
#pragma unroll
    for (int k = 0; k < 2 * NF - 3; ++k) pw *= xi;
    w = w * pw * w2 / w3 * ecm;
  }
  const double h = 0.5 * ecm;
  const int64_t L = 4 * nevt;
  mom[0 * nevt + i] = h; mom[1 * nevt + i] = 0.0; mom[2 * nevt + i] = 0.0; mom[3 * nevt + i] = h;
  mom[L + 0 * nevt + i] = h; mom[L + 1 * nevt + i] = 0.0; mom[L + 2 * nevt + i] = 0.0; mom[L + 3 * nevt + i] = -h;
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) mom[(int64_t)((2 + f) * 4 + mu) * nevt + i] = p[f][mu];
  wgt[i] = w;
}

cudaError_t launch_rambo(int nfinal, int64_t nevt, double ecm, const double* rnd, double* mom, double* wgt,
                         const RamboSetup& st, cudaStream_t s) {
  const int nt = 128;
  const int64_t grid = (nevt + nt - 1) / nt;
  switch (nfinal) {
    case 2: rambo_kernel<2><<<(unsigned)grid, nt, 0, s>>>(nevt, ecm, rnd, mom, wgt, st); break;
    case 3: rambo_kernel<3><<<(unsigned)grid, nt, 0, s>>>(nevt, ecm, rnd, mom, wgt, st); break;
    case 4: rambo_kernel<4><<<(unsigned)grid, nt, 0, s>>>(nevt, ecm, rnd, mom, wgt, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace mg
